"""Brute-force enumeration of local alignments (independent of any DP), for tiny inputs.

A local alignment is a start cell plus a sequence of operations: M (a_i with b_j), A (a_i with a
gap), B (b_j with a gap).  Its score is the sum of S over M operations minus g(k) for every
maximal run of k identical gap operations, g(k) = o + (k-1)e (mode 0) or o + k*e (mode 1).
The empty alignment scores 0.  Every alignment is enumerated explicitly.
"""


def gap_cost(k, o, e, mode):
    return o + (k - 1) * e if mode == 0 else o + k * e


def enumerate_alignments(a, b, S, o, e, mode):
    """Yield (score, i_s, i_e, j_s, j_e) for every alignment that starts and ends with M
    (1-based inclusive cells of its first and last M)."""
    m, n = len(a), len(b)

    def walk(i, j, score, run_op, run_len, first):
        # (i, j) = next unconsumed positions (0-based); the last op was M when run_len == 0
        if run_len == 0 and first is not None:
            yield (score, first[0] + 1, i, first[1] + 1, j)
        if i < m and j < n:
            s = score - (gap_cost(run_len, o, e, mode) if run_len else 0)
            yield from walk(i + 1, j + 1, s + int(S[a[i]][b[j]]), None, 0,
                            first if first is not None else (i, j))
        if first is None:
            return
        for op, di, dj in (("A", 1, 0), ("B", 0, 1)):
            if i + di > m or j + dj > n:
                continue
            if run_op == op:
                yield from walk(i + di, j + dj, score, op, run_len + 1, first)
            else:
                s = score - (gap_cost(run_len, o, e, mode) if run_len else 0)
                yield from walk(i + di, j + dj, s, op, 1, first)

    for i0 in range(m):
        for j0 in range(n):
            yield from walk(i0, j0, 0, None, 0, None)


def brute_best(a, b, S, o, e, mode):
    best = 0
    for al in enumerate_alignments(a, b, S, o, e, mode):
        best = max(best, al[0])
    return best


def brute_cells(a, b, S, o, e, mode):
    """(score, i_s, i_e, j_s, j_e): the end is the lexicographically smallest (i_e, j_e) among
    optimal alignments, the start the lexicographically largest (i_s, j_s) among the optimal
    alignments ending there.  All zero when the best score is 0."""
    als = list(enumerate_alignments(a, b, S, o, e, mode))
    best = max([0] + [x[0] for x in als])
    if best == 0:
        return (0, 0, 0, 0, 0)
    opt = [x for x in als if x[0] == best]
    ie, je = min((x[2], x[4]) for x in opt)
    i_s, j_s = max((x[1], x[3]) for x in opt if (x[2], x[4]) == (ie, je))
    return (best, i_s, ie, j_s, je)


def linear_gap_sw(a, b, S, g):
    """Textbook Smith-Waterman with a linear gap penalty g per gap residue (no E/F matrices)."""
    m, n = len(a), len(b)
    H = [[0] * (n + 1) for _ in range(m + 1)]
    best = 0
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            H[i][j] = max(0, H[i - 1][j - 1] + int(S[a[i - 1]][b[j - 1]]),
                          H[i - 1][j] - g, H[i][j - 1] - g)
            best = max(best, H[i][j])
    return best


def best_ungapped(a, b, S):
    """Best ungapped local segment: Kadane's maximum-subarray on every diagonal."""
    m, n = len(a), len(b)
    best = 0
    for d in range(-(m - 1), n):
        run = 0
        for i in range(m):
            j = i + d
            if 0 <= j < n:
                run = max(0, run + int(S[a[i]][b[j]]))
                best = max(best, run)
    return best
