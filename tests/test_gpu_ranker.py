"""GPU ranker kernels (BF16 tensor-core implicit GEMMs, FP32 accumulate) against the float64
oracle.  Tolerances follow from BF16 rounding: unit roundoff 2^-9 on every weight and stored
activation, three layers deep, gives ~1e-2 relative error; vectors and logits are checked at
3e-2 of their scale, gradients by per-tensor cosine >= 0.99 and relative norm error <= 6e-2."""
import numpy as np
import pytest

import oracle
from oracle import ranker as R
import paper_1908_10574_gb300 as cm
from paper_1908_10574_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return cm.Context(0)


def _set(rng_seed=7, n=10, lens=(1, 3, 8, 40, 129, 300, 511, 700, 1300, 60)):
    rng = np.random.default_rng(rng_seed)
    base = [synth.random_seq(rng, L) for L in lens[:n]]
    return synth.SeqSet.from_list(base)


def test_embeddings_match_oracle(ctx):
    ss = _set()
    p = R.init_params(11).astype(np.float32)
    ctx.ranker_set_params(p)
    got = ctx.ranker_embed(ss.seqs, ss.offsets)
    want = R.embed(ss.seqs, ss.offsets, p.astype(np.float64))
    for i in range(len(ss)):
        err = np.linalg.norm(got[i] - want[i]) / max(np.linalg.norm(want[i]), 1e-6)
        assert err < 3e-2, (i, err)


def test_empty_sequence_embeds_to_zero_and_logits(ctx):
    ss = synth.SeqSet.from_list([np.zeros(0, np.uint8), synth.random_seq(np.random.default_rng(1), 50)])
    p = R.init_params(12).astype(np.float32)
    ctx.ranker_set_params(p)
    got = ctx.ranker_embed(ss.seqs, ss.offsets)
    assert np.allclose(got[0], 0)
    z = ctx.ranker_logits(ss.seqs, ss.offsets, np.array([[0, 1], [1, 1], [1, 0]], np.int32))
    want = R.logits(ss.seqs, ss.offsets, p.astype(np.float64), [[0, 1], [1, 1], [1, 0]])
    assert np.allclose(z, want, rtol=3e-2, atol=3e-2 * np.abs(want).max())
    assert z[0] == z[2]


def test_loss_and_gradient_match_oracle(ctx):
    ss = _set(8, 10, (20, 35, 64, 90, 120, 150, 200, 260, 300, 33))
    rng = np.random.default_rng(3)
    pairs = rng.integers(0, len(ss), size=(24, 2)).astype(np.int32)
    labels = (rng.random(24) < 0.5).astype(np.float32)
    p = R.init_params(13).astype(np.float32)
    ctx.ranker_set_params(p)
    loss, grad = ctx.ranker_loss_grad(ss.seqs, ss.offsets, pairs, labels)
    wl, wg = R.loss_grad(ss.seqs, ss.offsets, p.astype(np.float64), pairs, labels)
    assert abs(loss - wl) <= 2e-2 * abs(wl)
    o = 0
    for name, shp in R.SHAPES:
        k = int(np.prod(shp))
        g, w = grad[o:o + k].astype(np.float64), wg[o:o + k]
        o += k
        nw = np.linalg.norm(w)
        if nw < 1e-9:
            continue
        cos = g @ w / (np.linalg.norm(g) * nw)
        rel = np.linalg.norm(g - w) / nw
        assert cos >= 0.99 and rel <= 6e-2, (name, cos, rel)


def test_training_learns_family_similarity(ctx):
    ss = synth.small_families()
    n = len(ss)
    pairs = oracle.triangle_pairs(n)
    scores = oracle.sw_batch(ss.seqs, ss.offsets, pairs, synth.BLOSUM62, 11, 1)
    y = (scores > 100).astype(np.float32)
    rng = np.random.default_rng(0)
    pos = np.nonzero(y == 1)[0]
    neg = rng.choice(np.nonzero(y == 0)[0], size=len(pos) * 3, replace=False)
    sel = rng.permutation(np.concatenate([pos, neg]))
    cut = int(0.8 * len(sel))
    tr, te = sel[:cut], sel[cut:]
    ctx.ranker_init(5)
    ctx.ranker_standardize(ss.seqs, ss.offsets, max_sample=200)
    V = ctx.ranker_embed(ss.seqs, ss.offsets)
    # zero mean / unit variance per channel up to BF16 cancellation (Z3 rows are stored in
    # BF16 while the channel mean being removed is large against its spread)
    assert np.abs(V.mean(0)).max() < 0.2 and np.abs(V.std(0, ddof=1) - 1).max() < 0.1
    z0 = ctx.ranker_logits(ss.seqs, ss.offsets, pairs[te])
    loss = ctx.ranker_train(ss.seqs, ss.offsets, pairs[tr], y[tr], epochs=6, batch_pairs=64,
                            lr=3e-4)
    z1 = ctx.ranker_logits(ss.seqs, ss.offsets, pairs[te])

    def auc(z, t):
        order = np.argsort(z)
        ranks = np.empty(len(z))
        ranks[order] = np.arange(1, len(z) + 1)
        npos = t.sum()
        return (ranks[t == 1].sum() - npos * (npos + 1) / 2) / (npos * (len(t) - npos))

    assert np.isfinite(loss)
    assert auc(z0, y[te]) > 0.75                 # standardised random features already rank
    assert auc(z1, y[te]) > 0.9 and auc(z1, y[te]) > auc(z0, y[te])


def test_ranked_merge_without_pruning_keeps_full_recall(ctx):
    ss = synth.small_families()
    ctx.ranker_init(9)
    ctx.ranker_standardize(ss.seqs, ss.offsets, max_sample=200)
    truth, _ = oracle.all_pairs(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, T=100)
    res = ctx.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, 100, 10 ** 6, 15,
                            use_ranker=True, prune_logit=-1e30)
    n = len(ss)
    assert res["stats"]["rep_comparisons"] == n * (n - 1) // 2
    assert res["stats"]["ranker_selected"] == n * (n - 1) // 2
    assert oracle.recall(res["pairs"], truth) == 1.0
    plain = ctx.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, 100, 10 ** 6, 15)
    assert res["pairs"].tolist() == plain["pairs"].tolist()


def test_trained_ranker_prunes_with_high_recall(ctx):
    """The learned path as the workload defines it: the ranker is trained on the set being
    clustered (pairs drawn inside groups of proteins, labelled by the GPU SW scores, one group
    per step), its pruning threshold is set to keep 99.8 % of held-out positives, and the
    ranked merge must keep the plain merge's recall to within 2 % while aligning fewer
    representative pairs."""
    import bench
    ss = synth.proteome(1600, family_size=8, singleton_frac=0.2, stream=12)
    rng = np.random.default_rng(4)
    pairs, _ = bench.grouped_training_pairs(ss.family, 40000, 50, rng)
    sc = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, synth.BLOSUM62, 11, 1)
    y = (sc > 100).astype(np.float32)
    cut = int(0.9 * len(pairs))
    ctx.ranker_init(3)
    ctx.ranker_standardize(ss.seqs, ss.offsets, max_sample=512)
    ctx.ranker_train(ss.seqs, ss.offsets, pairs[:cut], y[:cut], epochs=30, batch_pairs=25 * 50 + 64,
                     lr=1e-3, seed=5, flags=cm.CM_TRAIN_COMPONENTS | cm.CM_TRAIN_COSINE)
    z = ctx.ranker_logits(ss.seqs, ss.offsets, pairs[cut:])
    thr = float(np.quantile(z[y[cut:] == 1], 0.002))  # keep 99.8 % of held-out positives
    truth, _ = oracle.all_pairs(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, T=100)
    plain = ctx.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, 100, 138, 15)
    ranked = ctx.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, 100, 138, 15,
                               use_ranker=True, prune_logit=thr)
    rp, rr = oracle.recall(plain["pairs"], truth), oracle.recall(ranked["pairs"], truth)
    assert rr >= 0.98 * rp
    assert ranked["stats"]["rep_comparisons"] < 0.85 * plain["stats"]["rep_comparisons"]
    assert ranked["stats"]["comparisons_scored"] < plain["stats"]["comparisons_scored"]


def test_ranked_merge_prune_everything_large_matches_oracle(ctx):
    """A threshold above every logit prunes all pairs of merges at or above min_pairs; merges
    below it stay exact.  The oracle with keep = False reproduces this exactly."""
    ss = synth.small_families()
    n = len(ss)
    ctx.ranker_set_params(R.init_params(21).astype(np.float32))
    truth, scores = oracle.all_pairs(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, T=100)
    M = np.zeros((n, n), np.int64)
    M[np.triu_indices(n, 1)] = scores
    M = M + M.T
    for min_pairs in (4, 64, 1000):
        want = oracle.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, T=100, mT=138,
                                    mU=15, score_matrix=M, keep=lambda a, b: False,
                                    min_pairs=min_pairs)
        got = ctx.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, 100, 138, 15,
                                use_ranker=True, prune_logit=1e30, ranker_min_pairs=min_pairs)
        assert got["clusters"] == want["clusters"]
        assert got["pairs"].tolist() == want["pairs"].tolist()
        st, ws = got["stats"], want["stats"]
        assert (st["rep_comparisons"], st["exchange_comparisons"], st["intra_comparisons"]) == \
            (ws["rep"], ws["exchange"], ws["intra"])
        assert st["ranker_selected"] == 0


def _standardized_params(ss, seed):
    """Random ranker weights with the last conv layer rescaled so that every output channel
    of the sequence vectors has zero mean and unit variance over `ss` (float64, oracle side)."""
    flat = R.init_params(seed).astype(np.float32).astype(np.float64)
    p = R.unpack(flat)
    V = R.embed(ss.seqs, ss.offsets, flat)
    mu, sd = V.mean(0), V.std(0) + 1e-6
    p["W3"][...] = p["W3"] / sd[None, None, :]
    p["b3"][...] = (p["b3"] - mu) / sd
    return flat.astype(np.float32)


def test_ranked_merge_partial_pruning_matches_oracle(ctx):
    """A threshold inside the logit distribution selects part of every large merge's rep pairs
    (pair-mode lists of shared selections and single-query lists of the rest).  The oracle
    merge with keep = (its float64 logit >= threshold) must give the same clusters and pairs.
    The threshold is placed so that every pair within BF16 reach of it scores <= T: pruning
    such a pair or visiting it is the same `continue` in Algorithm 1, so only the
    rep-comparison count may differ, by at most the number of those pairs."""
    rng = np.random.default_rng(31)     # 4 families of 10 + 60 singletons: few significant pairs
    ss = synth.families(4, 10, rng.integers(60, 301, size=4), 31, singletons=60,
                        singleton_lengths=rng.integers(60, 301, size=60))
    n = len(ss)
    tri = oracle.triangle_pairs(n)
    truth, scores = oracle.all_pairs(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, T=100)
    M = np.zeros((n, n), np.int64)
    M[np.triu_indices(n, 1)] = scores
    M = M + M.T
    params = _standardized_params(ss, 7)
    z = R.logits(ss.seqs, ss.offsets, params.astype(np.float64), tri)
    Z = np.zeros((n, n))
    Z[tri[:, 0], tri[:, 1]] = z
    Z = Z + Z.T
    sig = M[tri[:, 0], tri[:, 1]] > 100
    band = 0.08
    cands = np.quantile(z, np.linspace(0.3, 0.7, 81))
    ok = [t for t in cands if not sig[np.abs(z - t) < band].any()]
    assert ok, "no threshold with only non-significant pairs near it"
    thr = float(ok[len(ok) // 2])
    ambiguous = int((np.abs(z - thr) < band).sum())
    want = oracle.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, T=100, mT=138, mU=15,
                                score_matrix=M, keep=lambda a, b: Z[a, b] >= thr, min_pairs=4)
    ctx.ranker_set_params(params)
    got = ctx.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, 100, 138, 15,
                            use_ranker=True, prune_logit=thr, ranker_min_pairs=4)
    assert got["clusters"] == want["clusters"]
    assert got["pairs"].tolist() == want["pairs"].tolist()
    st, ws = got["stats"], want["stats"]
    assert (st["exchange_comparisons"], st["intra_comparisons"]) == (ws["exchange"], ws["intra"])
    assert abs(st["rep_comparisons"] - ws["rep"]) <= ambiguous
    assert 0 < st["ranker_selected"] < n * (n - 1) // 2


def test_selection_kernel_keeps_the_pairs_above_threshold(ctx):
    """With full merges disabled every pair of sequences meets exactly once as a rep pair, so
    the tensor-core selection must keep exactly the pairs whose logit (computed by the separate
    head kernel) reaches the threshold -- up to pairs within BF16 error of it."""
    ss = synth.small_families()
    n = len(ss)
    ctx.ranker_init(4)
    ctx.ranker_standardize(ss.seqs, ss.offsets, max_sample=200)
    pairs = oracle.triangle_pairs(n)
    z = ctx.ranker_logits(ss.seqs, ss.offsets, pairs)
    thr = float(np.quantile(z, 0.7))
    res = ctx.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, 100, 10 ** 6, 15,
                            use_ranker=True, prune_logit=thr, ranker_min_pairs=0)
    st = res["stats"]
    want = int((z >= thr).sum())
    ambiguous = int((np.abs(z - thr) < 0.05).sum())
    assert abs(st["ranker_selected"] - want) <= ambiguous
    assert st["rep_comparisons"] == st["ranker_selected"]
    truth, _ = oracle.all_pairs(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, T=100)
    tset = {(int(i), int(j)) for i, j, _ in truth}
    assert all((int(i), int(j)) in tset for i, j, _ in res["pairs"])


def test_save_and_load_parameters(ctx, tmp_path):
    """Parameters written by ranker_save come back bit for bit, logits included; a file with a
    wrong tag or size is refused without touching the loaded parameters."""
    ss = _set()
    ctx.ranker_init(31)
    ctx.ranker_standardize(ss.seqs, ss.offsets, max_sample=64)
    p0 = ctx.ranker_get_params()
    pairs = np.array([[0, 1], [2, 3], [4, 5]], dtype=np.int32)
    z0 = ctx.ranker_logits(ss.seqs, ss.offsets, pairs)
    path = tmp_path / "ranker.bin"
    ctx.ranker_save(path)
    assert path.stat().st_size == 16 + 4 * ctx.ranker_num_params()
    ctx.ranker_init(32)
    assert not np.array_equal(ctx.ranker_get_params(), p0)
    ctx.ranker_load(path)
    assert np.array_equal(ctx.ranker_get_params(), p0)
    assert np.array_equal(ctx.ranker_logits(ss.seqs, ss.offsets, pairs), z0)
    bad = tmp_path / "bad.bin"
    bad.write_bytes(path.read_bytes()[:-4])
    with pytest.raises(cm.CMError):
        ctx.ranker_load(bad)
    assert np.array_equal(ctx.ranker_get_params(), p0)


def test_training_on_pair_groups_learns(ctx):
    """Pairs drawn inside groups of proteins (the benchmark's recipe) train one group per
    step with CM_TRAIN_COMPONENTS: every batch holds whole connected components of the pair
    graph, so each protein is
    embedded once per epoch.  The trained ranker must separate held-out pairs better than the
    standardised random one, and the step count must follow the groups."""
    import bench
    ss = synth.proteome(2400, family_size=8, singleton_frac=0.2, stream=14)
    rng = np.random.default_rng(6)
    pairs, gid = bench.grouped_training_pairs(ss.family, 24000, 48, rng)
    assert len(np.unique(gid)) >= 40
    sc = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, synth.BLOSUM62, 11, 1)
    y = (sc > 100).astype(np.float32)
    cut = int(0.9 * len(pairs))
    ctx.ranker_init(21)
    ctx.ranker_standardize(ss.seqs, ss.offsets, max_sample=512)
    z0 = ctx.ranker_logits(ss.seqs, ss.offsets, pairs[cut:])
    ctx.reset_stats()
    loss = ctx.ranker_train(ss.seqs, ss.offsets, pairs[:cut], y[:cut], epochs=30,
                            batch_pairs=15 * 48 + 64, lr=2e-3, seed=2,
                            flags=cm.CM_TRAIN_COMPONENTS | cm.CM_TRAIN_COSINE)
    launches = ctx.stats()["launches"]
    z1 = ctx.ranker_logits(ss.seqs, ss.offsets, pairs[cut:])

    def auc(z, t):
        order = np.argsort(z)
        ranks = np.empty(len(z))
        ranks[order] = np.arange(1, len(z) + 1)
        npos = t.sum()
        return (ranks[t == 1].sum() - npos * (npos + 1) / 2) / (npos * (len(t) - npos))

    assert np.isfinite(loss)
    a0, a1 = auc(z0, y[cut:]), auc(z1, y[cut:])
    assert a1 > max(a0 + 0.02, 0.89), (a0, a1)
    # one step per group (about 2,400 / 48 groups) per epoch, ~20 launches per step
    assert launches < 30 * 60 * 25
