"""Pins for the oracle ClusterMerge (Algorithm 1 Merge, Algorithm 2 BottomUpMerge).

Hand-traced cases use a mock similarity f (a table) and mock transitivity so that every branch
of Algorithm 1 (skip, absorb-and-break, absorb-and-continue, exchange, HasBeenMerged skip) is
pinned by an expected result written out by hand.  Real-sequence cases pin the special cases
the paper's argument fixes: with full merges disabled every similar pair is recovered (Sec. 3.3:
an element stays the representative of its own cluster, so every similar pair of
representatives meets and exchanges), and T = -1 makes every pair significant.
"""
import numpy as np
import pytest

import oracle
from oracle.cluster_merge import bottom_up_merge, intra_cluster_pairs, new_stats
from paper_1908_10574_gb300 import synth

T = 10


def run(n, F, trans):
    def score(x, y):
        return F[(min(x, y), max(x, y))]

    def transitive(r1, r2, s):
        return trans.get((r1, r2), (False, False))

    final, st = bottom_up_merge(n, score, transitive, T)
    return [(c.rep, list(c.objs)) for c in final], st


def test_n1_and_n2_branches():
    assert run(1, {}, {})[0] == [(0, [0])]
    # not similar: both clusters survive
    assert run(2, {(0, 1): 10}, {})[0] == [(0, [0]), (1, [1])]
    # cluster2 absorbs cluster1 (then break)
    assert run(2, {(0, 1): 11}, {(0, 1): (True, False)})[0] == [(1, [1, 0])]
    # cluster1 absorbs cluster2
    assert run(2, {(0, 1): 11}, {(0, 1): (False, True)})[0] == [(0, [0, 1])]
    # similar, not transitive: reps exchanged both ways
    assert run(2, {(0, 1): 11}, {})[0] == [(0, [0, 1]), (1, [1, 0])]


def test_n3_exchange_then_absorb():
    F = {(0, 1): 50, (0, 2): 40, (1, 2): 5}
    cl, st = run(3, F, {(2, 0): (True, False)})
    # merge(0,1): exchange -> C0=[0,1], C1=[1,0]; merge([C2],[C0,C1]): C0 absorbs C2, break
    assert cl == [(0, [0, 1, 2]), (1, [1, 0])]
    assert st["rep"] == 2 and st["exchange"] == 0 and st["full_merges"] == 1


def test_n3_absorb_continue_then_exchange_with_member_scoring():
    F = {(0, 1): 3, (0, 2): 30, (1, 2): 20}
    cl, st = run(3, F, {(2, 0): (False, True)})
    # merge(0,1): not similar -> [C0, C1]; merge([C2],[C0,C1]): C2 absorbs C0 (continue),
    # then exchange(C2, C1): member 0 of C2 scored against rep 1 (3 <= T, not added)
    assert cl == [(2, [2, 0, 1]), (1, [1, 2])]
    assert st["rep"] == 3 and st["exchange"] == 1


def test_n4_has_been_merged_skip():
    F = {(0, 1): 1, (2, 3): 2, (0, 2): 30, (0, 3): 4, (1, 3): 25, (1, 2): 99}
    cl, st = run(4, F, {(0, 2): (False, True), (1, 3): (True, False)})
    # merge(A=[C0,C1], B=[C2,C3]): C0 absorbs C2; C1 skips merged C2 (no comparison), then
    # C3 absorbs C1 and breaks
    assert cl == [(0, [0, 2]), (3, [3, 1])]
    assert st["rep"] == 5


def test_n4_full_chain_and_fifo_order():
    F = {(0, 1): 2, (2, 3): 40, (0, 2): 40, (1, 2): 40}
    cl, _ = run(4, F, {(2, 3): (False, True), (0, 2): (True, False), (1, 2): (False, True)})
    assert cl == [(1, [1, 2, 3, 0])]


def test_n5_fifo_pairs_leftover_with_next_result():
    # FIFO: (0,1)->A, (2,3)->B, (4,A)->C, (B,C)->final.  No similarity: singletons survive in
    # the order the merges append them.
    cl, st = run(5, {(i, j): 0 for i in range(5) for j in range(i + 1, 5)}, {})
    assert [r for r, _ in cl] == [2, 3, 4, 0, 1]
    assert st["merges"] == 4


def test_intra_cluster_pairs_dedup():
    class C:
        def __init__(self, objs):
            self.objs = objs
    st = new_stats()
    out = intra_cluster_pairs([C([3, 1, 2]), C([2, 1])], lambda x, y: 100 + x + y, T, st)
    assert out.tolist() == [[1, 2, 103], [1, 3, 104], [2, 3, 105]]
    assert st["intra"] == 3


@pytest.fixture(scope="module")
def small():
    ss = synth.small_families()
    S = synth.BLOSUM62
    truth, scores = oracle.all_pairs(ss.seqs, ss.offsets, S, 11, 1, T=60)
    n = len(ss)
    M = np.zeros((n, n), dtype=np.int64)
    iu = np.triu_indices(n, 1)
    M[iu] = scores
    M = M + M.T
    return ss, S, truth, M


def test_no_full_merges_gives_full_recall(small):
    ss, S, truth, M = small
    res = oracle.cluster_merge(ss.seqs, ss.offsets, S, 11, 1, T=60, mT=10 ** 9, mU=15,
                               score_matrix=M)
    assert res["stats"]["full_merges"] == 0
    assert len(res["clusters"]) == len(ss)
    assert oracle.recall(res["pairs"], truth) == 1.0


def test_negative_threshold_makes_every_pair_significant(small):
    ss, S, _, M = small
    n = len(ss)
    truth, _ = oracle.all_pairs(ss.seqs, ss.offsets, S, 11, 1, T=-1)
    assert len(truth) == n * (n - 1) // 2


def test_invariants_default_parameters(small):
    ss, S, truth, M = small
    res = oracle.cluster_merge(ss.seqs, ss.offsets, S, 11, 1, T=60, mT=83, mU=15,
                               score_matrix=M)
    covered = set()
    for rep, mem in res["clusters"]:
        assert mem[0] == rep and len(set(mem)) == len(mem)
        covered.update(mem)
    assert covered == set(range(len(ss)))
    tset = {(int(i), int(j)) for i, j, _ in truth}
    for i, j, s in res["pairs"]:
        assert i < j and (int(i), int(j)) in tset and s == M[i, j] and s > 60
    r = oracle.recall(res["pairs"], truth)
    assert 0.9 <= r <= 1.0
    assert res["stats"]["full_merges"] > 0


def test_lookup_and_direct_scoring_agree(small):
    ss, S, _, M = small
    sub = ss.subset(np.arange(40))
    Msub = M[:40, :40]
    a = oracle.cluster_merge(sub.seqs, sub.offsets, S, 11, 1, T=60, mT=83, mU=15,
                             score_matrix=Msub)
    b = oracle.cluster_merge(sub.seqs, sub.offsets, S, 11, 1, T=60, mT=83, mU=15)
    assert a["clusters"] == b["clusters"]
    assert a["pairs"].tolist() == b["pairs"].tolist()


def test_pruning_hook_keep_all_is_plain_and_keep_none_skips_large_merges():
    F = {(0, 1): 50, (0, 2): 40, (1, 2): 5, (0, 3): 12, (1, 3): 30, (2, 3): 3}
    plain, st = run(4, F, {})

    def score(x, y):
        return F[(min(x, y), max(x, y))]

    final, st2 = bottom_up_merge(4, score, lambda a, b, s: (False, False), T,
                                 keep=lambda a, b: True, min_pairs=0)
    assert [(c.rep, list(c.objs)) for c in final] == plain and st2["rep"] == st["rep"]
    # merges of two singletons (1 pair) stay exact below min_pairs=2; the final 2x2 merge is
    # pruned entirely, so no rep comparison happens there
    final, st3 = bottom_up_merge(4, score, lambda a, b, s: (False, False), T,
                                 keep=lambda a, b: False, min_pairs=2)
    assert st3["rep"] == 2
    assert [(c.rep, list(c.objs)) for c in final] == [(0, [0, 1]), (1, [1, 0]), (2, [2]), (3, [3])]


def run_partial(n, F, trans):
    def score(x, y):
        return F[(min(x, y), max(x, y))]

    def transitive(r1, r2, s):
        return trans.get((r1, r2), (False, False))

    final, st = bottom_up_merge(n, score, transitive, T, partial=True)
    return [(c.rep, list(c.objs)) for c in final], st


def test_partial_merges_see_set2_as_the_merge_began():
    """Sec. 5's partial merges, traced by hand on the case where the sequential merge skips a
    merged cluster (test_n4_has_been_merged_skip).  Merges (0,1) and (2,3): no similarity.
    Merge A=[C0,C1] with B=[C2,C3]: C0's partial merge absorbs C2 (t12) and skips C3 (4 <= T).
    C1's partial merge still sees C2 unmerged: f(1,2) = 99 > T, not transitive, so it
    exchanges the reps (C2's copy gains 1, C1 gains 2); then C3 absorbs C1 = [1, 2] (t21) and
    the loop breaks.  Result: C0 = [0, 2] and C3 = [3, 1, 2]; C2 was fully merged, so what C1
    added to it goes with it.  Visits: 1 + 1 + 2 + 2 = 6 (the sequential merge makes 5)."""
    F = {(0, 1): 1, (2, 3): 2, (0, 2): 30, (0, 3): 4, (1, 3): 25, (1, 2): 99}
    trans = {(0, 2): (False, True), (1, 3): (True, False)}
    cl, st = run_partial(4, F, trans)
    assert cl == [(0, [0, 2]), (3, [3, 1, 2])]
    assert st["rep"] == 6 and st["full_merges"] == 2 and st["exchanges"] == 1
    assert st["exchange"] == 0
    seq, st2 = run(4, F, trans)
    assert seq == [(0, [0, 2]), (3, [3, 1])] and st2["rep"] == 5


def test_partial_merges_exchange_members_of_the_snapshot_only():
    """A Set-2 cluster's members added by one partial merge are not scored by another.  Merges
    (0,1) and (2,3): no similarity.  Merge A=[C0,C1] with B=[C2,C3], f(0,2) = f(1,2) = 50, the
    rest <= T, no transitivity.  Sequentially, C0 exchanges with C2 (C2 = [2, 0], C0 = [0, 2]);
    then C1 exchanges with C2 = [2, 0]: rep 1 joins C2, and C2's member 0 is scored against
    rep 1 (f = 1: one exchange comparison, not added).  As partial merges, C1 sees C2 = [2]
    only, so 0 is never scored; C2 still ends as [2, 0, 1] from the two merges' additions."""
    F = {(0, 1): 1, (2, 3): 2, (0, 2): 50, (1, 2): 50, (0, 3): 3, (1, 3): 4}
    want = [(0, [0, 2]), (1, [1, 2]), (2, [2, 0, 1]), (3, [3])]
    seq, st_seq = run(4, F, {})
    par, st_par = run_partial(4, F, {})
    assert seq == want and par == want
    assert st_seq["exchange"] == 1 and st_par["exchange"] == 0
    assert st_seq["rep"] == st_par["rep"] == 6


def test_partial_merges_without_full_merges_give_full_recall(small):
    ss, S, truth, M = small
    res = oracle.cluster_merge(ss.seqs, ss.offsets, S, 11, 1, T=60, mT=10 ** 9, mU=15,
                               score_matrix=M, partial=True)
    assert res["stats"]["full_merges"] == 0
    assert oracle.recall(res["pairs"], truth) == 1.0
