"""Pins for the oracle's Smith-Waterman (Gotoh) scores and alignment cells (CPU only).

Each check ties the oracle to something other than itself: the published BLOSUM62 table's
facts, brute-force enumeration of all local alignments, closed forms (self-score, best
ungapped diagonal segment, textbook linear-gap SW), invariants, and hand-worked fixtures.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1908_10574_gb300 import synth
from tests.bruteforce import brute_best, brute_cells, linear_gap_sw, best_ungapped

S62 = synth.BLOSUM62.astype(np.int32)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sw_handworked.tsv")


def test_blosum62_published_facts():
    assert S62.shape == (20, 20)
    assert (S62 == S62.T).all()
    assert S62.min() == -4 and S62.max() == 11
    diag = dict(zip(synth.ALPHABET, np.diag(S62)))
    assert diag == dict(A=4, R=5, N=6, D=6, C=9, Q=5, E=5, G=6, H=8, I=4, L=4, K=5, M=5,
                        F=6, P=7, S=4, T=5, W=11, Y=7, V=4)
    # a few well-known off-diagonal entries
    ix = {c: i for i, c in enumerate(synth.ALPHABET)}
    assert S62[ix["I"], ix["V"]] == 3 and S62[ix["F"], ix["Y"]] == 3
    assert S62[ix["W"], ix["Y"]] == 2 and S62[ix["K"], ix["R"]] == 2
    assert S62[ix["W"], ix["N"]] == -4 and S62[ix["C"], ix["E"]] == -4


def _rand_case(rng, maxlen=4, alpha=3, asym=False):
    m, n = rng.integers(0, maxlen + 1, size=2)
    letters = rng.choice(20, size=alpha, replace=False)
    a = rng.choice(letters, size=m).astype(np.uint8)
    b = rng.choice(letters, size=n).astype(np.uint8)
    if asym:
        S = rng.integers(-6, 8, size=(20, 20)).astype(np.int32)
    else:
        S = S62
    return a, b, S


@pytest.mark.parametrize("mode", [0, 1])
def test_bruteforce_scores(mode):
    rng = np.random.default_rng(11 + mode)
    for trial in range(120):
        a, b, S = _rand_case(rng, maxlen=4, alpha=3, asym=(trial % 3 == 0))
        o = int(rng.integers(1, 9))
        e = int(rng.integers(0, o + 1))
        assert oracle.sw_score(a, b, S, o, e, mode) == brute_best(a, b, S, o, e, mode), \
            (synth.decode(a), synth.decode(b), o, e, mode)


@pytest.mark.parametrize("mode", [0, 1])
def test_bruteforce_cells(mode):
    rng = np.random.default_rng(21 + mode)
    for trial in range(80):
        a, b, S = _rand_case(rng, maxlen=4, alpha=3, asym=(trial % 2 == 0))
        o = int(rng.integers(1, 9))
        e = int(rng.integers(0, o + 1))
        assert oracle.sw_cells(a, b, S, o, e, mode) == brute_cells(a, b, S, o, e, mode), \
            (synth.decode(a), synth.decode(b), o, e, mode)


def test_bruteforce_length5_blosum():
    rng = np.random.default_rng(5)
    for _ in range(12):
        a = rng.integers(0, 20, size=5).astype(np.uint8)
        b = rng.integers(0, 20, size=4).astype(np.uint8)
        b[1] = a[2]
        assert oracle.sw_score(a, b, S62, 3, 1) == brute_best(a, b, S62, 3, 1, 0)


def test_golden_handworked():
    n = 0
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            f = line.rstrip("\n").split("\t")
            a, b = synth.encode(f[0]), synth.encode(f[1])
            o, e, mode, score = int(f[2]), int(f[3]), int(f[4]), int(f[5])
            assert oracle.sw_score(a, b, S62, o, e, mode) == score, line
            cells = oracle.sw_cells(a, b, S62, o, e, mode)
            assert cells[0] == score
            if f[6] != "-":
                assert cells[1:] == tuple(int(x) for x in f[6:10]), (line, cells)
            n += 1
    assert n >= 10


def test_self_score_closed_form():
    """For BLOSUM62, S(x,y) < (S(x,x)+S(y,y))/2 for x != y and every diagonal entry is
    positive, so any monotone matching of a with itself scores at most sum_i S(a_i,a_i)
    (each index is used at most once per side); the identity alignment attains it."""
    d = np.diag(S62)
    assert (d > 0).all()
    for x in range(20):
        for y in range(20):
            if x != y:
                assert 2 * S62[x, y] < d[x] + d[y]
    rng = np.random.default_rng(3)
    for _ in range(30):
        a = synth.random_seq(rng, int(rng.integers(1, 400)))
        assert oracle.sw_score(a, a, S62, 11, 1) == int(d[a].sum())


@pytest.mark.parametrize("mode", [0, 1])
def test_runs_split_by_a_gap_closed_form(mode):
    """a = x^n against b = x^p y^k x^q (n = p + q, S(x,y) < 0).  An alignment either stays
    inside one run of b (best S(x,x) max(p,q)) or crosses the y block; a crossing alignment
    that gaps g of the k y's (one gap: a second would only add an opening) pairs the other
    k - g with x's of a, so it has n - (k - g) x-x columns, k - g x-y columns and one gap of
    g, and every other crossing alignment drops positive x-x columns.  So the score is the
    largest of those counts' totals."""
    rng = np.random.default_rng(12 + mode)
    for _ in range(150):
        x = int(rng.integers(0, 20))
        ys = [y for y in range(20) if S62[x, y] < 0]
        y = int(rng.choice(ys))
        p, q, k = int(rng.integers(0, 13)), int(rng.integers(0, 13)), int(rng.integers(1, 9))
        o, e = [(11, 1), (5, 2), (3, 3), (1, 0), (20, 1)][int(rng.integers(0, 5))]
        n = p + q
        a = np.full(n, x, np.uint8)
        b = np.concatenate([np.full(p, x), np.full(k, y), np.full(q, x)]).astype(np.uint8)

        def gap(g):
            return 0 if g == 0 else (o + (g - 1) * e if mode == 0 else o + g * e)
        sxx, sxy = int(S62[x, x]), int(S62[x, y])
        cands = [sxx * max(p, q)]
        cands += [sxx * (n - k + g) + sxy * (k - g) - gap(g) for g in range(k + 1) if k - g <= n]
        assert oracle.sw_score(a, b, S62, o, e, mode) == max(cands), (x, y, p, q, k, o, e)
        assert oracle.sw_score(b, a, S62, o, e, mode) == max(cands)


def test_huge_gaps_reduce_to_best_ungapped_segment():
    rng = np.random.default_rng(4)
    for _ in range(40):
        a = synth.random_seq(rng, int(rng.integers(1, 60)))
        b = synth.random_seq(rng, int(rng.integers(1, 60)))
        if rng.random() < 0.5:
            b = np.concatenate([b, a[: len(a) // 2]])
        assert oracle.sw_score(a, b, S62, 10 ** 6, 10 ** 6) == best_ungapped(a, b, S62)


def test_equal_open_extend_is_linear_gap_sw():
    rng = np.random.default_rng(6)
    for _ in range(40):
        a = synth.random_seq(rng, int(rng.integers(1, 50)))
        b = synth.mutate(rng, a) if rng.random() < 0.7 else synth.random_seq(rng, 40)
        g = int(rng.integers(1, 8))
        assert oracle.sw_score(a, b, S62, g, g, 0) == linear_gap_sw(a, b, S62, g)


def test_blast_convention_equals_shifted_open():
    rng = np.random.default_rng(7)
    for _ in range(30):
        a = synth.random_seq(rng, int(rng.integers(1, 80)))
        b = synth.mutate(rng, a)
        assert oracle.sw_score(a, b, S62, 10, 1, 1) == oracle.sw_score(a, b, S62, 11, 1, 0)


def test_invariants_nonneg_symmetric_monotone():
    rng = np.random.default_rng(8)
    for _ in range(40):
        a = synth.random_seq(rng, int(rng.integers(1, 120)))
        b = synth.mutate(rng, a) if rng.random() < 0.5 else synth.random_seq(rng, 90)
        s = oracle.sw_score(a, b, S62, 11, 1)
        assert s >= 0
        assert s == oracle.sw_score(b, a, S62, 11, 1)
        ext = np.concatenate([synth.random_seq(rng, 7), a, synth.random_seq(rng, 5)])
        assert oracle.sw_score(ext, b, S62, 11, 1) >= s
    # empty inputs
    assert oracle.sw_score(np.zeros(0, np.uint8), a, S62, 11, 1) == 0
    assert oracle.sw_cells(np.zeros(0, np.uint8), a, S62, 11, 1) == (0, 0, 0, 0, 0)


def test_cells_describe_an_alignment_with_that_score():
    """The reported cells bound an optimal alignment: the local score of the two covered
    substrings equals the full score."""
    rng = np.random.default_rng(9)
    for _ in range(30):
        a = synth.random_seq(rng, int(rng.integers(20, 150)))
        b = synth.mutate(rng, a)
        sc, i_s, i_e, j_s, j_e = oracle.sw_cells(a, b, S62, 11, 1)
        assert sc > 0 and 1 <= i_s <= i_e <= len(a) and 1 <= j_s <= j_e <= len(b)
        assert oracle.sw_score(a[i_s - 1:i_e], b[j_s - 1:j_e], S62, 11, 1) == sc
        ua, ub = oracle.uncovered(len(a), len(b), (sc, i_s, i_e, j_s, j_e))
        assert ua == len(a) - (i_e - i_s + 1) and ub == len(b) - (j_e - j_s + 1)


def test_batch_matches_single_and_threshold_monotone():
    ss = synth.small_families()
    pairs = oracle.triangle_pairs(len(ss))[::97]
    sc = oracle.sw_batch(ss.seqs, ss.offsets, pairs, S62, 11, 1, threads=4)
    for k in range(0, len(pairs), 17):
        i, j = pairs[k]
        assert sc[k] == oracle.sw_score(ss[i], ss[j], S62, 11, 1)
    counts = [(sc > T).sum() for T in (20, 40, 60, 100, 200)]
    assert all(x >= y for x, y in zip(counts, counts[1:]))
