"""GPU ClusterMerge (device batches per merge round) against the oracle's plain sequential
Algorithms 1 and 2: clusters with their member order, the similar-pair set with scores, and the
logical comparison counts must be identical."""
import numpy as np
import pytest

import oracle
import paper_1908_10574_gb300 as cm
from paper_1908_10574_gb300 import synth

pytestmark = pytest.mark.gpu
S62 = synth.BLOSUM62


@pytest.fixture(scope="module")
def ctx():
    return cm.Context(0)


def _oracle_cm(ss, T, mT, mU):
    _, scores = oracle.all_pairs(ss.seqs, ss.offsets, S62, 11, 1, T=T)
    n = len(ss)
    M = np.zeros((n, n), np.int64)
    M[np.triu_indices(n, 1)] = scores
    M = M + M.T
    return oracle.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, T=T, mT=mT, mU=mU,
                                score_matrix=M)


def _check(got, want):
    assert got["clusters"] == want["clusters"]
    assert got["pairs"].tolist() == want["pairs"].tolist()
    st, ws = got["stats"], want["stats"]
    assert st["rep_comparisons"] == ws["rep"]
    assert st["exchange_comparisons"] == ws["exchange"]
    assert st["intra_comparisons"] == ws["intra"]
    assert st["full_merges"] == ws["full_merges"]
    assert st["exchanges"] == ws["exchanges"]
    assert st["merges"] == ws["merges"]


@pytest.mark.parametrize("T,mT,mU", [(100, 138, 15), (80, 110, 15), (60, 83, 15), (40, 83, 30),
                                     (60, 10 ** 6, 15), (-1, 150, 15)])
def test_small_families_exact(ctx, T, mT, mU):
    ss = synth.small_families()
    want = _oracle_cm(ss, T, mT, mU)
    got = ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, T, mT, mU)
    _check(got, want)


def test_tiny_sets_and_empty_sequences(ctx):
    rng = np.random.default_rng(1)
    root = synth.random_seq(rng, 120)
    cases = [[], [root], [root, synth.mutate(rng, root)],
             [root, np.zeros(0, np.uint8), synth.mutate(rng, root)],
             [synth.mutate(rng, root) for _ in range(7)]]
    for seqs in cases:
        ss = synth.SeqSet.from_list(seqs)
        want = _oracle_cm(ss, 60, 83, 15) if len(ss) > 1 else \
            oracle.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, T=60, mT=83, mU=15)
        got = ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, 60, 83, 15)
        _check(got, want)


def test_proteome_subset_with_singletons_exact_and_recall(ctx):
    full = synth.proteome(5000, family_size=8, singleton_frac=0.2, stream=7)
    ss = full.subset(np.arange(900))
    T, mT, mU = 100, 138, 15
    truth, scores = oracle.all_pairs(ss.seqs, ss.offsets, S62, 11, 1, T=T)
    n = len(ss)
    M = np.zeros((n, n), np.int64)
    M[np.triu_indices(n, 1)] = scores
    M = M + M.T
    want = oracle.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, T=T, mT=mT, mU=mU,
                                score_matrix=M)
    got = ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, T, mT, mU)
    _check(got, want)
    r = oracle.recall(got["pairs"], truth)
    assert r == oracle.recall(want["pairs"], truth)
    assert r > 0.998
    # the GPU's own all-against-all gives the same truth
    p, s = ctx.sw_allpairs(ss.seqs, ss.offsets, S62, 11, 1, T=T)
    assert sorted(zip(p[:, 0].tolist(), p[:, 1].tolist(), s.tolist())) == \
        sorted(map(tuple, truth.tolist()))


@pytest.mark.parametrize("T,mT,mU", [(100, 138, 15), (60, 10 ** 6, 15)])
def test_long_sequences_exact(ctx, T, mT, mU):
    """Tandem repeats of 4,500-7,000 residues among ordinary proteins: reps longer than the
    subject limit are scored as queries (rep waves and exchange waves), same-motif pairs
    overflow int16 and take the whole-CTA int32 path; results must not change."""
    base = synth.proteome(60, family_size=6, singleton_frac=0.3, stream=4)
    ss = synth.long_tail(base, 6, 2, stream=4, lo=4500, hi=7000)
    want = _oracle_cm(ss, T, mT, mU)
    got = ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, T, mT, mU)
    _check(got, want)



def test_empty_and_tiny_sequences_exact(ctx):
    """Empty and one-residue proteins among ordinary ones: their scores are 0, they never join
    a cluster by similarity, and the counts still match the sequential algorithm."""
    base = synth.proteome(50, family_size=5, singleton_frac=0.2, stream=6)
    rng = np.random.default_rng(6)
    seqs = [base[i] for i in range(len(base))]
    for k in (0, 7, 19, 33, 49):
        seqs.insert(k, np.zeros(0, np.uint8) if k % 2 == 0 else synth.random_seq(rng, 1))
    ss = synth.SeqSet.from_list(seqs)
    want = _oracle_cm(ss, 100, 138, 15)
    got = ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, 100, 138, 15)
    _check(got, want)
    ctx.ranker_init(5)                    # keeps every pair below: the weights do not matter
    ranked = ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, 100, 138, 15, use_ranker=True,
                               prune_logit=-1e30, ranker_min_pairs=0)
    assert ranked["clusters"] == want["clusters"]
    assert ranked["pairs"].tolist() == want["pairs"].tolist()


def test_transitivity_handworked_cases(ctx):
    """The hand-worked transitivity cases (Sec. 4, tests/golden/transitivity_handworked.tsv):
    the GPU merge takes the same full-merge branch as the hand derivation and the oracle, on
    the cells its own alignment-cells pass computes."""
    import test_oracle_transitivity as tt
    for case in tt.CASES:
        ss = synth.SeqSet.from_list([synth.encode(case["a"]), synth.encode(case["b"])])
        got = ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, tt.T, case["mT"], case["mU"])
        assert got["clusters"] == case["clusters"], case["why"]
        _check(got, _oracle_cm(ss, tt.T, case["mT"], case["mU"]))
        cells = ctx.sw_cells_batch(ss.seqs, ss.offsets, np.array([[0, 1]], np.int32), S62, 11, 1)
        assert tuple(cells[0]) == (case["score"],) + case["cells"], case["why"]


def test_checkpointed_run_matches_uninterrupted(ctx, tmp_path):
    """cluster_merge_resume stopping after every round (budget ~0), resumed from the state file
    until done: the same clusters, pairs and logical counts as the oracle's uninterrupted run,
    and the state of this problem is refused for other parameters."""
    ss = synth.proteome(600, family_size=6, singleton_frac=0.25, stream=5)
    T, mT, mU = 100, 138, 15
    want = _oracle_cm(ss, T, mT, mU)
    path = str(tmp_path / "cm.state")
    calls, got = 0, None
    while got is None and calls < 40:
        got = ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, T, mT, mU, state_path=path,
                                budget_seconds=1e-9)
        calls += 1
    assert got is not None and calls > 3        # one call per round boundary, then the finish
    _check(got, want)
    assert got["stats"]["rounds"] == calls
    with pytest.raises(cm.CMError):
        ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, T + 1, mT, mU, state_path=path)
