"""GPU alignments (sw_align_batch) against the oracle's traceback: the cells and every
run-length op must be identical (the span and the tie-breaking rule are both defined), on
family proteins (ties included), lognormal-length proteins, both gap conventions, an
asymmetric matrix, empty and unrelated pairs, long tandem repeats whose scores exceed the
int16 range, and the capacity error."""
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


def _check(ctx, ss, pairs, S, go, ge, flags=0, mode=0):
    cells, offs, runs = ctx.sw_align_batch(ss.seqs, ss.offsets, pairs, S, go, ge, flags=flags)
    assert offs[0] == 0 and offs[-1] == len(runs)
    for k, (x, y) in enumerate(pairs):
        wc, wops = oracle.sw_align(ss[x], ss[y], S, go, ge, mode)
        assert tuple(cells[k]) == wc, (k, x, y)
        got = [(int(v) >> 2, "MID"[int(v) & 3]) for v in runs[offs[k]:offs[k + 1]]]
        assert got == wops, (k, x, y, cm.ops_to_cigar(runs[offs[k]:offs[k + 1]]),
                             oracle.cigar(wops))
    return cells, offs, runs


def test_family_and_random_pairs_match_oracle(ctx):
    ss = synth.small_families()
    rng = np.random.default_rng(11)
    pairs = rng.integers(0, len(ss), size=(600, 2)).astype(np.int32)
    cells, _, _ = _check(ctx, ss, pairs, S62, 11, 1)
    assert (cells[:, 0] > 100).sum() > 20 and (cells[:, 0] < 40).sum() > 100


def test_lognormal_lengths_and_gap_conventions(ctx):
    rng = np.random.default_rng(12)
    roots = [synth.random_seq(rng, int(L)) for L in synth.lognormal_lengths(rng, 30, hi=1500)]
    seqs = []
    for r in roots:
        seqs += [r, synth.mutate(rng, r)]
    ss = synth.SeqSet.from_list(seqs)
    pairs = np.array([(2 * i, 2 * i + 1) for i in range(30)] +
                     [(2 * i + 1, 2 * i) for i in range(30)], dtype=np.int32)
    _check(ctx, ss, pairs, S62, 11, 1)
    _check(ctx, ss, pairs, S62, 10, 1, flags=cm.CM_GAP_BLAST, mode=1)
    _check(ctx, ss, pairs[:20], S62, 3, 3)


def test_asymmetric_matrix_ties_and_empty(ctx):
    rng = np.random.default_rng(13)
    S = rng.integers(-4, 6, size=(20, 20)).astype(np.int8)
    seqs = [np.zeros(0, np.uint8)] + [rng.integers(0, 4, rng.integers(1, 30)).astype(np.uint8)
                                      for _ in range(40)]
    ss = synth.SeqSet.from_list(seqs)
    pairs = np.array([(i, j) for i in range(len(ss)) for j in range(len(ss)) if (i * 7 + j) % 5 == 0],
                     dtype=np.int32)
    _check(ctx, ss, pairs, S, 4, 1)


def test_long_tandem_repeats(ctx):
    base = synth.proteome(4, family_size=2, stream=33)
    ss = synth.long_tail(base, 2, 1, stream=33, lo=4000, hi=5000)
    n = len(ss)
    pairs = np.array([(n - 2, n - 1), (n - 1, 0)], dtype=np.int32)
    cells, _, _ = _check(ctx, ss, pairs, S62, 11, 1)
    assert cells[0, 0] > 15000


def test_capacity_and_no_pairs(ctx):
    import ctypes
    from paper_1908_10574_gb300 import _lib
    ss = synth.small_families()
    pairs = np.array([[0, 1], [2, 3]], dtype=np.int32)
    cells = np.full((2, 5), -7, np.int32)
    offs = np.full(3, -7, np.int64)
    runs = np.full(1, -7, np.int32)
    total = ctypes.c_int64(0)
    m = np.ascontiguousarray(S62.reshape(-1))
    code = _lib.lib().sw_align_batch(ctx._h, ss.seqs.ctypes.data, ss.offsets.ctypes.data, len(ss),
                                     pairs.ctypes.data, 2, m.ctypes.data, 11, 1,
                                     cells.ctypes.data, offs.ctypes.data, runs.ctypes.data, 1,
                                     ctypes.byref(total), 0)
    assert code == -6 and total.value > 1
    assert (cells == -7).all() and (offs == -7).all() and (runs == -7).all()
    c2, o2, r2 = ctx.sw_align_batch(ss.seqs, ss.offsets, np.zeros((0, 2), np.int32), S62, 11, 1)
    assert c2.shape == (0, 5) and o2.tolist() == [0] and len(r2) == 0
