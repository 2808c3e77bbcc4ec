"""Oracle ClusterMerge: Algorithm 1 (Merge) and Algorithm 2 (BottomUpMerge), plain Python.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings of the paper taken here:
  * significance is f > T everywhere (Sec. 3 defines significant pairs by f(i, j) > T); the
    `continue` test of Algorithm 1 is therefore "s <= T".
  * the typo IsMerged in Algorithm 1 means HasBeenMerged.
  * cluster2.IsTransitive(cluster1)  <=>  s > mT and uncovered(rep1) < mU, where uncovered counts
    the residues of rep1 outside the optimal local alignment of (rep1, rep2) (Sec. 4, uA / uD);
    it absorbs cluster1 into cluster2.  cluster1.IsTransitive(cluster2) is the mirror image.
  * after cluster1 absorbs cluster2 the inner loop continues; after cluster2 absorbs cluster1 it
    breaks (Algorithm 1).
  * ExchangeSimilar(c1, c2) snapshots both member lists, scores every member m of c1 that is not
    already in c2 against rep2 (the pair (m, rep2)), adds it to c2 when the score is > T, then
    does the same for c2's snapshot against rep1.  The reps' own pair reuses s.  Members are
    de-duplicated within a cluster and kept in insertion order.
  * Algorithm 2's FIFO starts in input order and pops two sets at a time.
  * output: the union over final clusters of the intra-cluster pairs (i < j) with score > T
    (Sec. 6.1), sorted by (i, j).

Partial merges (Sec. 5): a merge of two large sets is split into partial merges, each merging
one cluster of Set 1 into (a subset of) Set 2 by Algorithm 1's inner loop; the distributed
runtime runs them on workers that never communicate, and its controller folds every returned
result into the merge's state -- elements added to existing clusters, fully merged clusters
marked -- and finally keeps the clusters of both sets that were not fully merged.
`merge_partial` follows that description: every cluster of Set 1 runs the inner loop against
Set 2 as it stood when the merge began (a worker's copy), the additions to each Set-2 cluster
are applied afterwards in Set-1 order (duplicates dropped), and a Set-2 cluster that some
partial merge fully merged is dropped together with whatever others added to it.
"""
from __future__ import annotations

from collections import deque

import numpy as np


class Cluster:
    """D1 of the paper's pseudocode: {rep, Objs, HasBeenMerged}."""

    __slots__ = ("rep", "objs", "members", "merged")

    def __init__(self, rep: int):
        self.rep = rep
        self.objs = [rep]
        self.members = {rep}
        self.merged = False

    def add(self, x: int):
        if x not in self.members:
            self.members.add(x)
            self.objs.append(x)

    def append_all(self, xs):
        for x in list(xs):
            self.add(x)


def exchange_similar(c1, c2, s, score, T, stats):
    snap1, snap2 = list(c1.objs), list(c2.objs)
    for m in snap1:
        if m in c2.members:
            continue
        if m == c1.rep:
            sm = s
        else:
            sm = score(m, c2.rep)
            stats["exchange"] += 1
        if sm > T:
            c2.add(m)
    for m in snap2:
        if m in c1.members:
            continue
        if m == c2.rep:
            sm = s
        else:
            sm = score(m, c1.rep)
            stats["exchange"] += 1
        if sm > T:
            c1.add(m)


def merge(cs1, cs2, score, transitive, T, stats, keep=None, min_pairs=0):
    """Algorithm 1.  `score(x, y)` is f on the pair (x, y); `transitive(r1, r2, s)` returns
    (cluster2.IsTransitive(cluster1), cluster1.IsTransitive(cluster2)) for reps r1, r2.
    Optional pruning (the learned ranker's role): when len(cs1)*len(cs2) >= min_pairs, a
    representative pair with keep(r1, r2) false is not compared at all."""
    prune = keep is not None and len(cs1) * len(cs2) >= min_pairs
    new_set = []
    for c1 in cs1:
        for c2 in cs2:
            if c2.merged:
                continue
            if prune and not keep(c1.rep, c2.rep):
                continue
            s = score(c1.rep, c2.rep)
            stats["rep"] += 1
            if s <= T:
                continue
            t21, t12 = transitive(c1.rep, c2.rep, s)
            if t21:
                c2.append_all(c1.objs)
                c1.merged = True
                stats["full_merges"] += 1
                break
            elif t12:
                c1.append_all(c2.objs)
                c2.merged = True
                stats["full_merges"] += 1
            else:
                exchange_similar(c1, c2, s, score, T, stats)
                stats["exchanges"] += 1
        if not c1.merged:
            new_set.append(c1)
    for c2 in cs2:
        if not c2.merged:
            new_set.append(c2)
    return new_set


def merge_partial(cs1, cs2, score, transitive, T, stats, keep=None, min_pairs=0):
    """Algorithm 1 as independent partial merges (Sec. 5, see the module docstring)."""
    prune = keep is not None and len(cs1) * len(cs2) >= min_pairs
    snap2 = [list(c2.objs) for c2 in cs2]          # Set 2 as the merge began
    added = [[] for _ in cs2]                       # what the partial merges add to each
    merged2 = [False] * len(cs2)
    new_set = []
    for c1 in cs1:
        for k, c2 in enumerate(cs2):
            if prune and not keep(c1.rep, c2.rep):
                continue
            s = score(c1.rep, c2.rep)
            stats["rep"] += 1
            if s <= T:
                continue
            t21, t12 = transitive(c1.rep, c2.rep, s)
            if t21:
                added[k].extend(c1.objs)
                c1.merged = True
                stats["full_merges"] += 1
                break
            elif t12:
                c1.append_all(snap2[k])
                merged2[k] = True
                stats["full_merges"] += 1
            else:
                view = Cluster(c2.rep)                  # the worker's copy of c2
                view.append_all(snap2[k])
                exchange_similar(c1, view, s, score, T, stats)
                added[k].extend(view.objs[len(snap2[k]):])
                stats["exchanges"] += 1
        if not c1.merged:
            new_set.append(c1)
    for k, c2 in enumerate(cs2):
        c2.append_all(added[k])
        if not merged2[k]:
            new_set.append(c2)
    return new_set


def bottom_up_merge(n, score, transitive, T, stats=None, keep=None, min_pairs=0,
                    partial=False):
    """Algorithm 2: FIFO of singleton cluster sets, pop two, merge, push, until one is left.
    With partial=True every merge runs as independent partial merges (merge_partial)."""
    merge_fn = merge_partial if partial else merge
    if stats is None:
        stats = new_stats()
    q = deque([Cluster(e)] for e in range(n))
    if not q:
        return [], stats
    while len(q) > 1:
        cs1 = q.popleft()
        cs2 = q.popleft()
        q.append(merge_fn(cs1, cs2, score, transitive, T, stats, keep, min_pairs))
        stats["merges"] += 1
    return q.popleft(), stats


def new_stats():
    return {"rep": 0, "exchange": 0, "intra": 0, "merges": 0, "full_merges": 0, "exchanges": 0}


def intra_cluster_pairs(clusters, score, T, stats):
    """Intra-cluster all-against-all (Sec. 6.1): every distinct pair (i < j) that shares a
    cluster is scored once; those with score > T are the similar pairs found."""
    seen = set()
    for c in clusters:
        mem = sorted(c.objs)
        for ii in range(len(mem)):
            for jj in range(ii + 1, len(mem)):
                seen.add((mem[ii], mem[jj]))
    out = []
    for (i, j) in sorted(seen):
        s = score(i, j)
        stats["intra"] += 1
        if s > T:
            out.append((i, j, s))
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def cluster_merge(seqs, offsets, S, gap_open, gap_extend, T, mT, mU, gap_mode=0,
                  score_matrix=None, keep=None, min_pairs=0, partial=False):
    """Full ClusterMerge over a sequence set: Algorithm 2 with protein transitivity (Sec. 4),
    then the intra-cluster all-against-all.  `score_matrix` (optional, n x n, from the oracle's
    own all_pairs) replaces direct SW calls by lookups; it is only used for symmetric S.

    Returns dict(clusters=[(rep, [members...]) ...], pairs=(k, 3) array, stats=dict)."""
    from . import sw_score, sw_cells, uncovered  # plain oracle SW

    S = np.asarray(S, dtype=np.int32)
    S = S.reshape(int(round(np.sqrt(S.size))), -1)
    n = len(offsets) - 1
    offsets = np.asarray(offsets, dtype=np.int64)
    seqs = np.asarray(seqs, dtype=np.uint8)

    def seq(x):
        return seqs[offsets[x]:offsets[x + 1]]

    symmetric = bool((S == S.T).all())
    if score_matrix is not None and symmetric:
        M = score_matrix

        def score(x, y):
            return int(M[x, y])
    else:
        def score(x, y):
            return sw_score(seq(x), seq(y), S, gap_open, gap_extend, gap_mode)

    def transitive(r1, r2, s):
        if not s > mT:
            return False, False
        a, b = seq(r1), seq(r2)
        cells = sw_cells(a, b, S, gap_open, gap_extend, gap_mode)
        uA, uB = uncovered(len(a), len(b), cells)
        return uA < mU, uB < mU

    final, stats = bottom_up_merge(n, score, transitive, T, keep=keep, min_pairs=min_pairs,
                                   partial=partial)
    pairs = intra_cluster_pairs(final, score, T, stats)
    clusters = [(c.rep, list(c.objs)) for c in final]
    return {"clusters": clusters, "pairs": pairs, "stats": stats}
