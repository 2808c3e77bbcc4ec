"""Pins of the oracle incremental greedy clustering (the paper's comparison method, Sec. 2,
restated in oracle/greedy.py): a hand-traced case on a mock similarity, and the special cases
its definition fixes -- with full representation impossible (mT = inf) every sequence becomes
a representative, so all pairs are compared and recall is exactly 1; with every pair similar
and represented (T = mT = -1) everything joins the first sequence's cluster."""
import numpy as np

import oracle
from oracle.greedy import greedy, greedy_cluster
from paper_1908_10574_gb300 import synth


def test_hand_traced_greedy():
    F = {(0, 1): 50, (0, 2): 5, (1, 2): 40, (0, 3): 60, (1, 3): 5, (2, 3): 45}
    unc = {(3, 0): 3}

    def score(x, r):
        return F[(min(x, r), max(x, r))]

    # x=0 starts C0.  x=1: f(1,0) = 50 > T joins C0, 50 <= mT so it starts C1.  x=2: f(2,0) <= T,
    # f(2,1) = 40 joins C1, starts C2.  x=3: f(3,0) = 60 > mT with 3 uncovered < mU = 5:
    # represented by C0 (joins it); f(3,1) <= T; f(3,2) = 45 joins C2; starts nothing.
    cl, st = greedy(4, score, lambda x, r: unc.get((x, r), 100), T=10, mT=55, mU=5)
    assert [(c.rep, c.objs) for c in cl] == [(0, [0, 1, 3]), (1, [1, 2]), (2, [2, 3])]
    assert st["rep"] == 0 + 1 + 2 + 3
    # the same with 5 uncovered residues (not < mU): 3 becomes a representative too
    unc[(3, 0)] = 5
    cl, st = greedy(4, score, lambda x, r: unc.get((x, r), 100), T=10, mT=55, mU=5)
    assert [(c.rep, c.objs) for c in cl] == [(0, [0, 1, 3]), (1, [1, 2]), (2, [2, 3]), (3, [3])]


def test_no_representation_compares_all_pairs_with_full_recall():
    ss = synth.small_families()
    n = len(ss)
    truth, scores = oracle.all_pairs(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, T=60)
    M = np.zeros((n, n), np.int64)
    M[np.triu_indices(n, 1)] = scores
    M = M + M.T
    res = greedy_cluster(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, T=60, mT=10 ** 9, mU=15,
                         score_matrix=M)
    assert len(res["clusters"]) == n
    assert res["stats"]["rep"] == n * (n - 1) // 2
    assert oracle.recall(res["pairs"], truth) == 1.0
    # default thresholds: a real clustering, found pairs are true pairs
    res = greedy_cluster(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, T=60, mT=83, mU=15,
                         score_matrix=M)
    assert len(res["clusters"]) < n and res["stats"]["rep"] < n * (n - 1) // 2
    tset = {(int(i), int(j)) for i, j, _ in truth}
    assert all((int(i), int(j)) in tset for i, j, _ in res["pairs"])
    assert 0.9 <= oracle.recall(res["pairs"], truth) <= 1.0


def test_everything_similar_and_represented_makes_one_cluster():
    ss = synth.small_families().subset(np.arange(30))
    res = greedy_cluster(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, T=-1, mT=-1, mU=10 ** 6)
    assert res["clusters"] == [(0, list(range(30)))]
    assert res["stats"]["rep"] == 29
    assert len(res["pairs"]) == 30 * 29 // 2
