"""GPU parity of the Smith-Waterman path against the CPU oracle (exact integer equality).

Every test calls the CUDA path through the C ABI (ctypes binding) and the oracle on the same
seeded inputs.  Sizes span several query tiles (R bins), multi-pass queries (> 1024 residues),
ragged tails, empty and 1-residue sequences, int16 saturation (int32 rerun), both gap
conventions and an asymmetric matrix.
"""
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


def _lognormal_set(n, stream, hi=5000):
    rng = np.random.default_rng(stream)
    lens = synth.lognormal_lengths(rng, n, hi=hi)
    return synth.SeqSet.from_list([synth.random_seq(rng, int(L)) for L in lens])


def test_small_allpairs_scores_exact(ctx):
    ss = synth.small_families()
    pairs = oracle.triangle_pairs(len(ss))
    got = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    assert np.array_equal(got, want)


def test_random_pairs_lognormal_exact(ctx):
    ss = _lognormal_set(600, 1)
    pairs = synth.random_pairs(len(ss), 4000, stream=5)
    got = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    assert np.array_equal(got, want)


def test_long_queries_multipass_and_ragged(ctx):
    rng = np.random.default_rng(2)
    lens = [1, 2, 31, 32, 33, 127, 128, 129, 1023, 1024, 1025, 1100, 2049, 3000, 4999]
    seqs = [synth.random_seq(rng, L) for L in lens]
    # homologous partners so scores are large and alignments long
    seqs += [synth.mutate(rng, s) for s in seqs]
    ss = synth.SeqSet.from_list(seqs)
    n = len(ss)
    pairs = np.array([(i, j) for i in range(n) for j in range(n)], dtype=np.int32)
    got = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    assert np.array_equal(got, want)


def _every_tile_set(stream):
    """Two queries per register-tile width R = 1..32 (32R-20 and 32R-3 residues, so the
    length-sorted pairing puts both in tile R) plus short sequences of every length mod 4.
    Every other sequence starts with a substituted copy of an earlier one, so scores are
    large and optimal alignments cross lanes."""
    rng = np.random.default_rng(stream)
    lens = [1, 2, 3, 5, 6, 7] + [L for R in range(1, 33) for L in (max(32 * R - 20, 12), 32 * R - 3)]
    seqs = []
    for i, L in enumerate(lens):
        s = synth.random_seq(rng, L)
        if i % 2 and i > 6:
            donor = synth.mutate(rng, seqs[int(rng.integers(6, i))], sub_rate=0.2, indel_rate=0.0)
            k = min(L, len(donor))
            s[:k] = donor[:k]
        seqs.append(s)
    return synth.SeqSet.from_list(seqs)


def test_every_tile_width_pair_mode_exact(ctx):
    """All pairs through the all-against-all path: query pairs share a tile (pair mode) at
    every R = 1..32, odd and even."""
    ss = _every_tile_set(21)
    got_pairs, got_scores = ctx.sw_allpairs(ss.seqs, ss.offsets, S62, 11, 1, -1)
    tri = oracle.triangle_pairs(len(ss))
    want = oracle.sw_batch(ss.seqs, ss.offsets, tri, S62, 11, 1)
    got = {(min(int(i), int(j)), max(int(i), int(j))): int(v)
           for (i, j), v in zip(np.asarray(got_pairs), np.asarray(got_scores))}
    assert len(got) == len(tri)
    assert all(got[(int(i), int(j))] == int(w) for (i, j), w in zip(tri, want))


def test_every_tile_width_single_query_mode_exact(ctx):
    """Every ordered pair through sw_score_batch: each sequence is a lone query (single-query,
    two-stream mode) at every R = 1..32."""
    ss = _every_tile_set(22)
    n = len(ss)
    pairs = np.array([(i, j) for i in range(n) for j in range(n) if i != j], dtype=np.int32)
    got = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    assert np.array_equal(got, want)


def test_long_tail_tandem_repeats_exact(ctx):
    """Long tandem repeats sharing a motif align over their whole length with scores far above
    the int16 range (int32 rerun); pairs with short proteins and across motifs stay small."""
    base = synth.proteome(30, family_size=10, stream=9)
    ss = synth.long_tail(base, 6, 2, stream=9, lo=8000, hi=12000)
    n = len(ss)
    longs = list(range(30, n))
    pairs = np.array([(i, j) for i in longs for j in longs if i < j] +
                     [(i, j) for i in longs for j in range(0, 30, 7)], dtype=np.int32)
    got = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    assert np.array_equal(got, want)
    assert (want > 32767).sum() >= 6                  # same-motif pairs overflow int16
    st = ctx.stats()
    assert st["saturated"] > 0
    # the same pairs through the all-against-all path (significant set and scores)
    p, s = ctx.sw_allpairs(ss.seqs, ss.offsets, S62, 11, 1, 100)
    tri = oracle.triangle_pairs(n)
    sel = np.isin(tri[:, 0], longs) | np.isin(tri[:, 1], longs)
    ws = oracle.sw_batch(ss.seqs, ss.offsets, tri[sel], S62, 11, 1)
    want_sig = {(int(i), int(j)): int(v) for (i, j), v in zip(tri[sel], ws) if v > 100}
    got_sig = {(int(i), int(j)): int(v) for (i, j), v in zip(np.asarray(p), np.asarray(s))
               if int(i) in longs or int(j) in longs}
    assert got_sig == want_sig
    # alignment cells of long pairs (whole-CTA pipeline: >= 2,048 columns, >= 512 rows),
    # same-motif and cross-motif, both orientations, plus long x short
    cp = np.array([(longs[0], longs[2]), (longs[2], longs[0]), (longs[1], longs[3]),
                   (longs[0], longs[1]), (longs[4], 3), (5, longs[5])], dtype=np.int32)
    cells = ctx.sw_cells_batch(ss.seqs, ss.offsets, cp, S62, 11, 1)
    for k, (x, y) in enumerate(cp):
        assert tuple(cells[k]) == oracle.sw_cells(ss[x], ss[y], S62, 11, 1), (k, x, y)


def test_empty_sequences(ctx):
    rng = np.random.default_rng(3)
    seqs = [np.zeros(0, np.uint8), synth.random_seq(rng, 50), np.zeros(0, np.uint8),
            synth.random_seq(rng, 1)]
    ss = synth.SeqSet.from_list(seqs)
    pairs = np.array([(i, j) for i in range(4) for j in range(4)], dtype=np.int32)
    got = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    assert np.array_equal(got, want)
    assert len(ctx.sw_score_batch(ss.seqs, ss.offsets, np.zeros((0, 2), np.int32), S62, 11, 1)) == 0


def test_int16_saturation_rerun_exact(ctx):
    rng = np.random.default_rng(4)
    w = synth.encode("W" * 3100)                      # self score 34100 > int16
    motif = synth.tandem_repeat(rng, 6000)             # self-similar, large scores
    seqs = [w, w[:2900], motif, synth.mutate(rng, motif), synth.random_seq(rng, 300)]
    ss = synth.SeqSet.from_list(seqs)
    pairs = np.array([(i, j) for i in range(5) for j in range(5)], dtype=np.int32)
    ctx.reset_stats()
    got = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    assert want.max() > 32767
    assert np.array_equal(got, want)
    assert ctx.stats()["saturated"] > 0


@pytest.mark.parametrize("mode", [0, 1])
def test_gap_conventions_and_asymmetric_matrix(ctx, mode):
    rng = np.random.default_rng(10 + mode)
    S = rng.integers(-5, 9, size=(20, 20)).astype(np.int8)
    ss = _lognormal_set(120, 20 + mode, hi=1500)
    pairs = synth.random_pairs(len(ss), 800, stream=7 + mode)
    flags = cm.CM_GAP_BLAST if mode else 0
    got = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S, 7, 2, flags=flags)
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs, S, 7, 2, gap_mode=mode)
    assert np.array_equal(got, want)


def test_force_int32_path_exact(ctx):
    ss = _lognormal_set(200, 30, hi=2500)
    pairs = synth.random_pairs(len(ss), 600, stream=9)
    got = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1, flags=cm.CM_FORCE_INT32)
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    assert np.array_equal(got, want)


def test_device_pointer_path(ctx):
    import torch
    ss = synth.small_families()
    pairs = oracle.triangle_pairs(len(ss))[::7].copy()
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    got = ctx.sw_score_batch(d(ss.seqs), d(ss.offsets), d(pairs), d(S62.reshape(-1)), 11, 1)
    torch.cuda.synchronize()
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    assert np.array_equal(got.cpu().numpy(), want)


def test_allpairs_significant_set(ctx):
    ss = synth.small_families()
    truth, scores = oracle.all_pairs(ss.seqs, ss.offsets, S62, 11, 1, T=60)
    p, s = ctx.sw_allpairs(ss.seqs, ss.offsets, S62, 11, 1, T=60)
    got = sorted(zip(p[:, 0].tolist(), p[:, 1].tolist(), s.tolist()))
    assert got == sorted(map(tuple, truth.tolist()))
    # every pair significant at T = -1, scores exact
    p, s = ctx.sw_allpairs(ss.seqs, ss.offsets, S62, 11, 1, T=-1, capacity=1 << 15)
    n = len(ss)
    assert len(p) == n * (n - 1) // 2
    M = np.zeros((n, n), np.int64)
    M[np.triu_indices(n, 1)] = scores
    assert np.array_equal(s, M[p[:, 0], p[:, 1]])


def test_allpairs_parts_union(ctx):
    ss = _lognormal_set(300, 40, hi=3000)
    truth, _ = oracle.all_pairs(ss.seqs, ss.offsets, S62, 11, 1, T=35)
    got = []
    for part in range(5):
        p, s = ctx.sw_allpairs(ss.seqs, ss.offsets, S62, 11, 1, T=35, part=part, n_parts=5)
        got += list(zip(p[:, 0].tolist(), p[:, 1].tolist(), s.tolist()))
    assert sorted(got) == sorted(map(tuple, truth.tolist()))


def test_cells_match_oracle(ctx):
    ss = synth.small_families()
    rng = np.random.default_rng(12)
    pairs = synth.random_pairs(len(ss), 300, stream=12)
    fam = ss.family
    same = np.nonzero(fam[:, None] == fam[None, :])
    pick = rng.choice(len(same[0]), 200, replace=False)
    pairs = np.concatenate([pairs, np.stack([same[0][pick], same[1][pick]], 1)]).astype(np.int32)
    got = ctx.sw_cells_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    for k, (a, b) in enumerate(pairs):
        assert tuple(got[k]) == oracle.sw_cells(ss[a], ss[b], S62, 11, 1), (k, a, b)


def test_invalid_residue_and_arguments(ctx):
    ss = synth.small_families()
    bad = ss.seqs.copy()
    bad[5] = 25
    with pytest.raises(cm.CMError) as ei:
        ctx.sw_score_batch(bad, ss.offsets, np.array([[0, 1]], np.int32), S62, 11, 1)
    assert ei.value.code == -2
    with pytest.raises(cm.CMError) as ei:
        ctx.sw_score_batch(ss.seqs, ss.offsets, np.array([[0, 999]], np.int32), S62, 11, 1)
    assert ei.value.code == -1
    with pytest.raises(cm.CMError):
        ctx.sw_score_batch(ss.seqs, ss.offsets, np.array([[0, 1]], np.int32), S62, 0, 1)


def test_ascii_input(ctx):
    txt = ["HEAGAWGHEE", "PAWHEAE", "mkwvtfisll"]
    seqs = np.frombuffer("".join(txt).encode(), np.uint8)
    off = np.cumsum([0] + [len(t) for t in txt]).astype(np.int64)
    got = ctx.sw_score_batch(seqs, off, np.array([[0, 1], [2, 2]], np.int32), S62, 11, 1,
                             flags=cm.CM_ASCII)
    assert got.tolist() == [17, 52]


def test_autotune_choice_cache_and_unchanged_scores(ctx, tmp_path):
    ss = _lognormal_set(400, 50, hi=2000)
    pairs = synth.random_pairs(len(ss), 500, stream=13)
    before = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    cache = str(tmp_path / "tune.txt")
    w, r = ctx.autotune(ss.seqs, ss.offsets, S62, 11, 1, sample_seqs=300, cache_path=cache)
    assert w in (4, 8, 16) and r in (4096, 8192, 16384, 32768)
    assert open(cache).read().split()[1:] == [str(w), str(r)]
    ctx.set_tuning(4, 4096)
    assert ctx.autotune(ss.seqs, ss.offsets, S62, 11, 1, cache_path=cache) == (w, r)
    after = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    assert np.array_equal(before, after)
    assert np.array_equal(after, oracle.sw_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1))


def test_full_size_allpairs_sampled_exact(ctx):
    """The all-against-all of 20,000 proteome-shaped proteins in the autotuned launch
    configuration and the 16-part split the benchmark times.  Checked on a 100,000-pair random
    sample (significant exactly when the oracle scores > T, with the same score) and on the
    scores of every significant pair near or above the int16 range plus 5,000 others."""
    ss = synth.proteome(20000, 10)
    n = len(ss)
    ctx.autotune(ss.seqs, ss.offsets, S62, 11, 1, sample_seqs=3000)
    sig = {}
    for part in range(16):
        p, s = ctx.sw_allpairs(ss.seqs, ss.offsets, S62, 11, 1, 100, part, 16, capacity=1 << 20)
        sig.update({(int(i), int(j)): int(v) for (i, j), v in zip(p, s)})
    rng = np.random.default_rng(2020)
    a = rng.integers(0, n, 120000)
    b = rng.integers(0, n, 120000)
    keep = a != b
    pairs = np.unique(np.stack([np.minimum(a, b), np.maximum(a, b)], 1)[keep], axis=0)[:100000]
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs.astype(np.int32), S62, 11, 1)
    for (i, j), w in zip(pairs, want):
        if w > 100:
            assert sig.get((int(i), int(j))) == int(w), (i, j, w)
        else:
            assert (int(i), int(j)) not in sig, (i, j, w)
    keys = np.array(list(sig.keys()), dtype=np.int32)
    vals = np.array(list(sig.values()))
    pick = np.concatenate([np.flatnonzero(vals >= 32767 - 11),
                           rng.choice(len(keys), 5000, replace=False)])
    assert np.array_equal(oracle.sw_batch(ss.seqs, ss.offsets, keys[pick], S62, 11, 1), vals[pick])


def test_full_size_single_query_modes_sampled_exact(ctx):
    """sw_score_batch's single-query launch modes at full size.  A generic pair list becomes
    one block per distinct first sequence, a lone query that runs with two or four subject
    streams per warp (the modes that score a ranked merge's per-representative subject
    lists).  64 queries of the 20,000-protein set, spread over its length range (short ones
    in 16-lane segments, long ones in 512-column passes), each against every protein: 1.28M
    pairs, checked on a 100,000-pair sample and on every pair the oracle scores above T."""
    ss = synth.proteome(20000, 10)
    n = len(ss)
    order = np.argsort(ss.lengths, kind="stable")
    queries = order[np.linspace(0, n - 1, 64).astype(np.int64)]
    assert ss.lengths[queries].min() <= 256 and ss.lengths[queries].max() > 1024
    pairs = np.stack([np.repeat(queries, n), np.tile(np.arange(n), len(queries))], 1)
    pairs = pairs[pairs[:, 0] != pairs[:, 1]].astype(np.int32)
    got = ctx.sw_score_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    rng = np.random.default_rng(2021)
    pick = rng.choice(len(pairs), 100000, replace=False)
    want = oracle.sw_batch(ss.seqs, ss.offsets, pairs[pick], S62, 11, 1)
    assert np.array_equal(got[pick], want)
    # every planted relative of a query (same family) plus every pair the GPU puts above T
    fam = ss.family
    rel = np.flatnonzero((fam[pairs[:, 0]] == fam[pairs[:, 1]]) & (fam[pairs[:, 0]] >= 0))
    hi = np.union1d(rel, np.flatnonzero(got > 100))
    assert len(hi) > 64
    assert np.array_equal(got[hi], oracle.sw_batch(ss.seqs, ss.offsets, pairs[hi], S62, 11, 1))


def test_long_pair_wait_limit_times_out_then_recovers(ctx):
    """The whole-CTA long-pair kernel's one device wait (a column pass waiting for the rows
    of the pass before it) is bounded.  With a limit of one poll the later passes cannot see
    their predecessor's first 32 rows in time, so the call must return CM_ERR_TIMEOUT with
    nothing written; with the default limit restored the same context gives the oracle's
    cells."""
    base = synth.proteome(4, family_size=2, stream=31)
    ss = synth.long_tail(base, 2, 1, stream=31, lo=6000, hi=7000)
    x, y = len(ss) - 2, len(ss) - 1
    pairs = np.array([(x, y)], dtype=np.int32)
    out = np.full((1, 5), -7, dtype=np.int32)
    ctx.set_wait_limit(1)
    try:
        with pytest.raises(cm.CMError) as ei:
            ctx.sw_cells_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1, out=out)
        assert ei.value.code == -5
        assert out.tolist() == [[-7] * 5]
    finally:
        ctx.set_wait_limit(0)
    cells = ctx.sw_cells_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1)
    assert tuple(cells[0]) == oracle.sw_cells(ss[x], ss[y], S62, 11, 1)
    assert cells[0][0] > 10000
