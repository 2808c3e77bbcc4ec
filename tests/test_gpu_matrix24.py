"""GPU parity with 24 x 24 matrices over ARNDCQEGHILKMFPSTWYVBZX* (CM_MATRIX24): BLOSUM62 and
PAM250 with B, Z, X and * in the sequences, exact against the oracle -- random pairs over
many tile widths and both launch modes, multi-pass queries, int16 saturation with the int32
rerun on long tandem repeats, alignment cells and traceback, ASCII input, and ClusterMerge
under PAM250 with the paper's thresholds (T = 181, mT = 250, mU = 15, Sec. 4, Sec. 6.1)."""
import numpy as np
import pytest

import oracle
import paper_1908_10574_gb300 as cm
from paper_1908_10574_gb300 import synth

pytestmark = pytest.mark.gpu
B24, P24 = synth.BLOSUM62_24, synth.PAM250_24


@pytest.fixture(scope="module")
def ctx():
    return cm.Context(0)


def _with_extra_letters(rng, codes, rate=0.05):
    out = codes.copy()
    m = rng.random(len(out)) < rate
    out[m] = rng.integers(20, 24, size=int(m.sum()))
    return out


def _set(n, stream, hi=1400):
    rng = np.random.default_rng(stream)
    lens = np.concatenate([np.arange(1, 40, 3), synth.lognormal_lengths(rng, n, hi=hi)])
    roots = [_with_extra_letters(rng, synth.random_seq(rng, int(L))) for L in lens]
    seqs = []
    for r in roots:
        seqs += [r, _with_extra_letters(rng, synth.mutate(rng, r[r < 20]) if (r < 20).any() else r)]
    return synth.SeqSet.from_list(seqs)


@pytest.mark.parametrize("S", [B24, P24], ids=["BLOSUM62_24", "PAM250_24"])
def test_scores_match_oracle(ctx, S):
    ss = _set(80, 71)
    rng = np.random.default_rng(3)
    n = len(ss)
    pairs = np.concatenate([np.stack([np.arange(0, n, 2), np.arange(1, n, 2)], 1),
                            rng.integers(0, n, size=(3000, 2))]).astype(np.int32)
    got = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S, 11, 1)
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs, S, 11, 1)
    assert np.array_equal(got, want)
    # one query against many subjects: the single-query modes
    one = np.stack([np.full(n, 5), np.arange(n)], 1).astype(np.int32)
    assert np.array_equal(ctx.sw_score_batch(ss.seqs, ss.offsets, one, S, 11, 1),
                          oracle.sw_batch(ss.seqs, ss.offsets, one, S, 11, 1))
    blast = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs[:500], S, 10, 1, flags=cm.CM_GAP_BLAST)
    assert np.array_equal(blast, oracle.sw_batch(ss.seqs, ss.offsets, pairs[:500], S, 10, 1, 1))


def test_long_tandem_repeats_int32_and_cells(ctx):
    rng = np.random.default_rng(8)
    motif = _with_extra_letters(rng, synth.random_seq(rng, 40), 0.2)
    # long enough that the same-motif pair scores above the int16 range (int32 rescoring)
    longs = [synth.tandem_repeat(rng, int(L), motif=motif) for L in (11000, 12500)]
    ss = synth.SeqSet.from_list(longs + [_with_extra_letters(rng, synth.random_seq(rng, 300))])
    pairs = np.array([(0, 1), (1, 0), (0, 2), (2, 1)], dtype=np.int32)
    got = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, P24, 11, 1)
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs, P24, 11, 1)
    assert np.array_equal(got, want) and want.max() > 32767
    cells = ctx.sw_cells_batch(ss.seqs, ss.offsets, pairs, P24, 11, 1)
    for k, (x, y) in enumerate(pairs):
        assert tuple(cells[k]) == oracle.sw_cells(ss[x], ss[y], P24, 11, 1)


def test_alignments_ascii_and_rejections(ctx):
    ss = _set(20, 72, hi=400)
    rng = np.random.default_rng(4)
    pairs = rng.integers(0, len(ss), size=(200, 2)).astype(np.int32)
    cells, offs, runs = ctx.sw_align_batch(ss.seqs, ss.offsets, pairs, B24, 11, 1)
    for k, (x, y) in enumerate(pairs):
        wc, wops = oracle.sw_align(ss[x], ss[y], B24, 11, 1)
        assert tuple(cells[k]) == wc
        assert cm.ops_to_cigar(runs[offs[k]:offs[k + 1]]) == oracle.cigar(wops)
    text = "".join(synth.decode(ss[i]) for i in range(len(ss)))
    asc = np.frombuffer(text.lower().encode(), dtype=np.uint8)
    got = ctx.sw_score_batch(asc, ss.offsets, pairs, B24, 11, 1, flags=cm.CM_ASCII)
    assert np.array_equal(got, oracle.sw_batch(ss.seqs, ss.offsets, pairs, B24, 11, 1))
    # a 20 x 20 matrix does not accept B, Z, X, *
    with pytest.raises(cm.CMError) as ei:
        ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, synth.BLOSUM62, 11, 1)
    assert ei.value.code == -2


def test_cluster_merge_pam250_paper_thresholds(ctx):
    rng = np.random.default_rng(9)
    base = synth.families(30, 8, rng.integers(150, 400, size=30), stream=73)
    seqs = [_with_extra_letters(rng, base[i], 0.02) for i in range(len(base))]
    ss = synth.SeqSet.from_list(seqs)
    n = len(ss)
    truth, scores = oracle.all_pairs(ss.seqs, ss.offsets, P24, 11, 1, T=181)
    M = np.zeros((n, n), np.int64)
    M[np.triu_indices(n, 1)] = scores
    M = M + M.T
    want = oracle.cluster_merge(ss.seqs, ss.offsets, P24, 11, 1, T=181, mT=250, mU=15,
                                score_matrix=M)
    got = ctx.cluster_merge(ss.seqs, ss.offsets, P24, 11, 1, 181, 250, 15)
    assert got["clusters"] == want["clusters"]
    assert got["pairs"].tolist() == want["pairs"].tolist()
    assert got["stats"]["rep_comparisons"] == want["stats"]["rep"]
    assert want["stats"]["full_merges"] > 0 and len(truth) > 100
