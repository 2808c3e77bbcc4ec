"""Pins of the oracle's alignment traceback (one optimal local alignment per pair, as
run-length ops): hand-worked alignments from tests/golden/align_handworked.tsv, including a
tie the preference rule decides, and invariants that hold for any input -- the ops rescore to
the Smith-Waterman score, consume exactly the span of the alignment cells, and start and end
with an aligned pair -- on random proteins and tiny inputs, both gap conventions and an
asymmetric matrix.  The rescoring here is written independently of the oracle's DP."""
import os

import numpy as np
import pytest

import oracle
from paper_1908_10574_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
S62 = synth.BLOSUM62


def golden():
    out = []
    for line in open(os.path.join(HERE, "golden", "align_handworked.tsv")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.rstrip("\n").split("\t")
        out.append((f[0], f[1], int(f[2]), int(f[3]), int(f[4]), int(f[5]), f[6], f[7]))
    return out


@pytest.mark.parametrize("case", golden(), ids=lambda c: "%s/%s/%d" % (c[0], c[1], c[4]))
def test_handworked_alignments(case):
    a, b, go, ge, mode, score, ops, why = case
    cells, got = oracle.sw_align(synth.encode(a), synth.encode(b), S62, go, ge, mode)
    assert cells[0] == score, why
    assert oracle.cigar(got) == ops, why


def rescore(a, b, S, go, ge, mode, cells, ops):
    """Score of the alignment the ops describe, from its definition: matrix entries of the
    aligned pairs minus the cost of every gap run (k residues cost go + (k-1) ge, or
    go + k ge in the BLAST convention).  Also checks the ops cover the span exactly."""
    _, i_s, i_e, j_s, j_e = cells
    i, j, total = i_s - 1, j_s - 1, 0
    for n, op in ops:
        if op == "M":
            for _ in range(n):
                total += int(S[a[i], b[j]])
                i += 1
                j += 1
        else:
            total -= go + (n - 1) * ge if mode == 0 else go + n * ge
            if op == "I":
                i += n
            else:
                j += n
    assert (i, j) == (i_e, j_e)
    return total


def check_pair(a, b, S, go, ge, mode):
    cells, ops = oracle.sw_align(a, b, S, go, ge, mode)
    if cells[0] == 0:
        assert ops == []
        return
    assert ops[0][1] == "M" and ops[-1][1] == "M"
    assert all(ops[k][1] != ops[k + 1][1] for k in range(len(ops) - 1))   # maximal runs
    assert rescore(a, b, S, go, ge, mode, cells, ops) == cells[0]
    assert cells[0] == oracle.sw_score(a, b, S, go, ge, mode)


def test_invariants_on_proteins():
    ss = synth.small_families()
    rng = np.random.default_rng(3)
    for _ in range(150):
        x, y = rng.integers(0, len(ss), 2)
        for go, ge, mode in ((11, 1, 0), (10, 1, 1), (4, 4, 0)):
            check_pair(ss[x], ss[y], S62, go, ge, mode)


def test_invariants_on_tiny_inputs_and_asymmetric_matrix():
    rng = np.random.default_rng(4)
    S = rng.integers(-6, 7, size=(20, 20))
    for _ in range(600):
        a = rng.integers(0, 4, rng.integers(1, 9)).astype(np.uint8)
        b = rng.integers(0, 4, rng.integers(1, 9)).astype(np.uint8)
        go, ge = int(rng.integers(1, 8)), 0
        ge = int(rng.integers(0, go + 1))
        check_pair(a, b, S, go, ge, int(rng.integers(0, 2)))
