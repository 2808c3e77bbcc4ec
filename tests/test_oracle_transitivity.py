"""Pins of the oracle's protein-transitivity closure (Sec. 4) on real sequences.

The closure decides Algorithm 1's two full-merge branches from the representatives' score and
the residues their optimal local alignment leaves uncovered.  Each case of
tests/golden/transitivity_handworked.tsv was worked out by hand from the BLOSUM62 table (the
derivation is in its last column): the alignment cells, the uncovered counts of both
representatives, both transitivity tests and the merge result.  Together they catch swapped
operands (uA for uB), an inclusive bound on either side (<= mU, >= mT) and an uncovered count
that looks at one end of the representative only.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1908_10574_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
S62 = synth.BLOSUM62
T = 20


def load_cases():
    out = []
    for line in open(os.path.join(HERE, "golden", "transitivity_handworked.tsv")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.rstrip("\n").split("\t")
        clusters = []
        for part in f[13].split("|"):
            rep, mem = part.split(":")
            clusters.append((int(rep), [int(x) for x in mem.split(",")]))
        out.append(dict(a=f[0], b=f[1], mT=int(f[2]), mU=int(f[3]), score=int(f[4]),
                        cells=tuple(int(x) for x in f[5:9]), uA=int(f[9]), uB=int(f[10]),
                        t21=bool(int(f[11])), t12=bool(int(f[12])), clusters=clusters,
                        why=f[14]))
    return out


CASES = load_cases()


def test_fixture_is_complete():
    assert len(CASES) == 9
    # every branch of the closure appears: absorb either way, and the exchange
    kinds = {len(c["clusters"]) for c in CASES} | {c["clusters"][0][0] for c in CASES}
    assert kinds == {0, 1, 2}


@pytest.mark.parametrize("case", CASES, ids=[c["why"][:40] for c in CASES])
def test_cells_and_uncovered(case):
    a, b = synth.encode(case["a"]), synth.encode(case["b"])
    cells = oracle.sw_cells(a, b, S62, 11, 1)
    assert cells == (case["score"],) + case["cells"], case["why"]
    assert oracle.uncovered(len(a), len(b), cells) == (case["uA"], case["uB"])


@pytest.mark.parametrize("case", CASES, ids=[c["why"][:40] for c in CASES])
def test_transitivity_and_merge_result(case):
    ss = synth.SeqSet.from_list([synth.encode(case["a"]), synth.encode(case["b"])])
    res = oracle.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, T=T, mT=case["mT"],
                               mU=case["mU"])
    assert res["clusters"] == case["clusters"], case["why"]
    st = res["stats"]
    assert st["rep"] == 1 and st["exchange"] == 0
    assert st["full_merges"] == int(case["t21"] or case["t12"])
    assert st["exchanges"] == int(not (case["t21"] or case["t12"]))
    # the pair is similar (score > T) and shares a final cluster either way
    assert res["pairs"].tolist() == [[0, 1, case["score"]]]
