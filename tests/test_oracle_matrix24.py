"""Pins of the 24-letter path of the oracle (matrices over ARNDCQEGHILKMFPSTWYVBZX*): the
published tables as entered (symmetry, ranges, the diagonals everyone quotes, the 20 x 20
block of BLOSUM62 unchanged), and brute-force enumeration of every local alignment on tiny
inputs drawn from B, Z, X, * and a few amino acids, under both tables and both gap
conventions, with the cells' tie-break."""
import numpy as np
import pytest

import oracle
from paper_1908_10574_gb300 import synth
from bruteforce import enumerate_alignments


def brute_best(a, b, S, o, e, mode):
    return max([0] + [x[0] for x in enumerate_alignments(a, b, S, o, e, mode)])


def test_tables_as_published():
    B, P = synth.BLOSUM62_24.astype(int), synth.PAM250_24.astype(int)
    for M in (B, P):
        assert M.shape == (24, 24) and (M == M.T).all()
    assert (B[:20, :20] == synth.BLOSUM62).all()
    assert B.min() == -4 and B.max() == 11 and (B[23, :23] == -4).all() and B[23, 23] == 1
    assert [B[k, k] for k in range(20, 23)] == [4, 4, -1]                  # B, Z, X
    assert P.min() == -8 and P.max() == 17 and (P[23, :23] == -8).all() and P[23, 23] == 1
    diag = dict(zip(synth.ALPHABET, [2, 6, 2, 4, 12, 4, 4, 5, 6, 5, 6, 5, 6, 9, 6, 2, 3, 17, 10, 4]))
    assert all(P[k, k] == diag[ch] for k, ch in enumerate(synth.ALPHABET))
    # B pools D and N, Z pools E and Q: their rows stay within the pooled rows' range
    for pooled, parts in ((20, (2, 3)), (21, (5, 6))):
        lo = np.minimum(P[parts[0], :20], P[parts[1], :20])
        hi = np.maximum(P[parts[0], :20], P[parts[1], :20])
        assert ((P[pooled, :20] >= lo - 1) & (P[pooled, :20] <= hi + 1)).all()
    assert synth.decode(synth.encode("ACBZX*", alphabet24=True)) == "ACBZX*"
    with pytest.raises(ValueError):
        synth.encode("ACB")


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("table", ["BLOSUM62_24", "PAM250_24"])
def test_bruteforce_with_extra_letters(table, mode):
    S = getattr(synth, table)
    rng = np.random.default_rng(24 + mode)
    letters = np.array([0, 2, 3, 20, 21, 22, 23], dtype=np.uint8)   # A N D B Z X *
    for _ in range(100):
        a = rng.choice(letters, size=int(rng.integers(1, 5))).astype(np.uint8)
        b = rng.choice(letters, size=int(rng.integers(1, 5))).astype(np.uint8)
        o = int(rng.integers(1, 9))
        e = int(rng.integers(0, o + 1))
        want = brute_best(a, b, S, o, e, mode)
        assert oracle.sw_score(a, b, S, o, e, mode) == want
        cells = oracle.sw_cells(a, b, S, o, e, mode)
        assert cells[0] == want
        if want > 0:
            firsts = sorted((x[2], x[4]) for x in enumerate_alignments(a, b, S, o, e, mode)
                            if x[0] == want)
            assert (cells[2], cells[4]) == firsts[0]              # first end cell, row-major
