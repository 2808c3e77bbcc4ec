"""Oracle incremental greedy clustering, plain Python.  TEST INFRASTRUCTURE ONLY (see
oracle/__init__.py).

The comparison method the paper measures ClusterMerge against (Sec. 2, after Wittwer et al.)
is an iterative greedy clustering that builds clusters around representatives one sequence at
a time: a sequence similar to a representative goes into that cluster; a sequence similar to
no representative starts a new cluster as its representative.  The paper states that its
transitivity function is built the same way as this method's (Sec. 4).  Restated here:

  for each sequence x in input order:
      compare x with every representative r in creation order (a logical comparison each);
      x joins the cluster of every r with f(x, r) > T;
      x is represented when some r has f(x, r) > mT and fewer than mU residues of x lie
      outside their optimal local alignment (the Sec. 4 test, x in the absorbed role);
      an x that no representative represents becomes a new representative (its own cluster).

The output is the same as ClusterMerge's: the intra-cluster all-against-all over the final
clusters (Sec. 6.1), pairs (i < j) with f > T.
"""
from __future__ import annotations

import numpy as np

from .cluster_merge import intra_cluster_pairs, new_stats


class GreedyCluster:
    __slots__ = ("rep", "objs")

    def __init__(self, rep):
        self.rep = rep
        self.objs = [rep]


def greedy(n, score, uncovered_x, T, mT, mU, stats=None):
    """Clusters (representatives in creation order, members in joining order, rep first).
    `score(x, r)` is f; `uncovered_x(x, r)` the residues of x outside the optimal local
    alignment of (x, r).  stats["rep"] counts comparisons with representatives,
    stats["full_merges"] the sequences an existing cluster represents."""
    if stats is None:
        stats = new_stats()
    clusters = []
    for x in range(n):
        represented = False
        for c in list(clusters):
            s = score(x, c.rep)
            stats["rep"] += 1
            if s <= T:
                continue
            c.objs.append(x)
            if s > mT and uncovered_x(x, c.rep) < mU:
                represented = True
        if not represented:
            clusters.append(GreedyCluster(x))
        else:
            stats["full_merges"] += 1          # represented by an existing cluster
    return clusters, stats


def greedy_cluster(seqs, offsets, S, gap_open, gap_extend, T, mT, mU, gap_mode=0,
                   score_matrix=None):
    """Greedy clustering of a sequence set plus the intra-cluster all-against-all.  Returns
    dict(clusters=[(rep, [members...]) ...], pairs=(k, 3) array, stats=dict)."""
    from . import sw_score, sw_cells, uncovered

    S = np.asarray(S, dtype=np.int32)
    S = S.reshape(int(round(np.sqrt(S.size))), -1)
    n = len(offsets) - 1
    offsets = np.asarray(offsets, dtype=np.int64)
    seqs = np.asarray(seqs, dtype=np.uint8)

    def seq(x):
        return seqs[offsets[x]:offsets[x + 1]]

    if score_matrix is not None and bool((S == S.T).all()):
        M = score_matrix

        def score(x, y):
            return int(M[x, y])
    else:
        def score(x, y):
            return sw_score(seq(x), seq(y), S, gap_open, gap_extend, gap_mode)

    def uncovered_x(x, r):
        a, b = seq(x), seq(r)
        return uncovered(len(a), len(b), sw_cells(a, b, S, gap_open, gap_extend, gap_mode))[0]

    final, stats = greedy(n, score, uncovered_x, T, mT, mU)
    pairs = intra_cluster_pairs(final, score, T, stats)
    return {"clusters": [(c.rep, list(c.objs)) for c in final], "pairs": pairs, "stats": stats}
