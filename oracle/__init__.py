"""CPU oracle for the batched Smith-Waterman / ClusterMerge path.

TEST INFRASTRUCTURE ONLY: only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline
leg may import this package.  The product path never calls it, and it shares no code with the
CUDA path (the only common module is the seeded input generator, which holds no arithmetic of
the method).

Contents
  * ``sw_score`` / ``sw_batch`` / ``sw_cells`` -- plain scalar Gotoh DP in C (``sw_oracle.c``),
    int64 arithmetic; the paper's similarity f (Sec. 4).
  * ``all_pairs`` -- the all-against-all ground truth and its significant pairs f > T (Sec. 3).
  * ``cluster_merge`` -- Algorithm 1 (Merge) and Algorithm 2 (BottomUpMerge) in plain Python,
    followed by the intra-cluster all-against-all (Sec. 6.1).  See ``oracle/cluster_merge.py``.
  * ``ranker`` -- float64 forward/backward of the representative ranker (``oracle/ranker.py``).

Pins (tests/test_oracle_*.py) tie every function to something other than itself: brute-force
enumeration of local alignments, closed forms (self-score, Kadane on diagonals, linear-gap
textbook SW), invariants, hand-worked fixtures under tests/golden/, and hand-checked
ClusterMerge traces.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_sw_oracle.so")
_lib_handle = None


def build(force: bool = False) -> str:
    """Compile sw_oracle.c with gcc (plain C, -O2, no target-specific flags)."""
    src = os.path.join(_HERE, "sw_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.cm_oracle_sw.restype = i64
        lib.cm_oracle_sw.argtypes = [p, i64, p, i64, p, i64, i64, ctypes.c_int]
        lib.cm_oracle_sw_cells.restype = None
        lib.cm_oracle_sw_cells.argtypes = [p, i64, p, i64, p, i64, i64, ctypes.c_int, p]
        lib.cm_oracle_sw_align.restype = i64
        lib.cm_oracle_sw_align.argtypes = [p, i64, p, i64, p, i64, i64, ctypes.c_int, p, p, i64]
        lib.cm_oracle_sw_batch.restype = ctypes.c_int
        lib.cm_oracle_sw_batch.argtypes = [p, p, p, i64, p, i64, i64, ctypes.c_int, p,
                                           ctypes.c_int]
        _lib_handle = lib
    return _lib_handle


def _matrix(S):
    """The 24 x 24 int32 table the C code reads: a 24 x 24 matrix as given, a 20 x 20 one in
    its top-left corner (rows and columns of B, Z, X, * unused then)."""
    S = np.asarray(S, dtype=np.int32)
    k = int(round(np.sqrt(S.size)))
    assert k * k == S.size and k in (20, 24), "matrix must be 20 x 20 or 24 x 24"
    out = np.zeros((24, 24), dtype=np.int32)
    out[:k, :k] = S.reshape(k, k)
    return np.ascontiguousarray(out)


def _codes(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint8))


def sw_score(a, b, S, gap_open, gap_extend, gap_mode=0) -> int:
    """Smith-Waterman (Gotoh) score of residue-code arrays a, b; S[x, y] = score(a_i=x, b_j=y)."""
    a, b, S = _codes(a), _codes(b), _matrix(S)
    return int(_lib().cm_oracle_sw(a.ctypes.data, len(a), b.ctypes.data, len(b), S.ctypes.data,
                                   int(gap_open), int(gap_extend), int(gap_mode)))


def sw_cells(a, b, S, gap_open, gap_extend, gap_mode=0):
    """(score, i_start, i_end, j_start, j_end), 1-based inclusive cells of the optimal local
    alignment chosen by the tie-break: end = first row-major cell with H = score; start = the
    first row-major cell of the same DP on the reversed prefixes (the alignment ending at the
    end cell that spans the fewest residues of a, then of b).  All zero when score == 0."""
    a, b, S = _codes(a), _codes(b), _matrix(S)
    out = np.zeros(5, dtype=np.int64)
    _lib().cm_oracle_sw_cells(a.ctypes.data, len(a), b.ctypes.data, len(b), S.ctypes.data,
                              int(gap_open), int(gap_extend), int(gap_mode), out.ctypes.data)
    return tuple(int(v) for v in out)


OPS = "MID"


def sw_align(a, b, S, gap_open, gap_extend, gap_mode=0):
    """One optimal local alignment: (cells, ops) with cells as sw_cells and ops a list of
    (run length, op) from start to end, op 'M' (a_i with b_j), 'I' (a_i against a gap) or 'D'
    (b_j against a gap).  The span is sw_cells'; inside it the global affine alignment of the
    two substrings, traced back from the end preferring M, then I, then D, and a gap's
    opening over its extension."""
    a, b, S = _codes(a), _codes(b), _matrix(S)
    cells = np.zeros(5, dtype=np.int64)
    cap = len(a) + len(b) + 1
    ops = np.zeros(cap, dtype=np.int32)
    k = _lib().cm_oracle_sw_align(a.ctypes.data, len(a), b.ctypes.data, len(b), S.ctypes.data,
                                  int(gap_open), int(gap_extend), int(gap_mode),
                                  cells.ctypes.data, ops.ctypes.data, cap)
    assert k >= 0
    return tuple(int(v) for v in cells), [(int(x) >> 2, OPS[int(x) & 3]) for x in ops[:k]]


def cigar(ops):
    """CIGAR text of run-length ops, e.g. [(3, 'M'), (1, 'I')] -> '3M1I'."""
    return "".join("%d%s" % (n, op) for n, op in ops)


def uncovered(a_len, b_len, cells):
    """Residues of a and of b outside the chosen optimal local alignment (Sec. 4, uA / uD)."""
    score, i_s, i_e, j_s, j_e = cells
    if score == 0:
        return a_len, b_len
    return a_len - (i_e - i_s + 1), b_len - (j_e - j_s + 1)


def sw_batch(seqs, offsets, pairs, S, gap_open, gap_extend, gap_mode=0, threads=None):
    """Scores of pairs[k] = (a, b) over a concatenated code array; int64 results."""
    seqs = _codes(seqs)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    S = _matrix(S)
    out = np.zeros(len(pairs), dtype=np.int64)
    if threads is None:
        threads = os.cpu_count() or 1
    if len(pairs):
        _lib().cm_oracle_sw_batch(seqs.ctypes.data, offsets.ctypes.data, pairs.ctypes.data,
                                  len(pairs), S.ctypes.data, int(gap_open), int(gap_extend),
                                  int(gap_mode), out.ctypes.data, int(threads))
    return out


def triangle_pairs(n):
    """All pairs (i, j), i < j, in row-major order of i then j."""
    i, j = np.triu_indices(n, k=1)
    return np.stack([i, j], axis=1).astype(np.int32)


def all_pairs(seqs, offsets, S, gap_open, gap_extend, T, gap_mode=0, threads=None):
    """All-against-all ground truth (Sec. 1 / Sec. 6.1): every pair i < j is aligned and the
    significant pairs f(i, j) > T (Sec. 3) are returned as an (k, 3) int64 array (i, j, score)
    sorted by (i, j), together with the full score vector in triangle order."""
    n = len(offsets) - 1
    pairs = triangle_pairs(n)
    scores = sw_batch(seqs, offsets, pairs, S, gap_open, gap_extend, gap_mode, threads)
    keep = scores > T
    sig = np.concatenate([pairs[keep].astype(np.int64), scores[keep, None]], axis=1)
    return sig, scores


def recall(found, truth):
    """|found ∩ truth| / |truth| over (i, j) pairs (Sec. 6.1); 1.0 when truth is empty."""
    t = {(int(i), int(j)) for i, j in np.asarray(truth)[:, :2]} if len(truth) else set()
    f = {(int(i), int(j)) for i, j in np.asarray(found)[:, :2]} if len(found) else set()
    if not t:
        return 1.0
    return len(t & f) / len(t)


from .cluster_merge import cluster_merge, merge, bottom_up_merge, Cluster  # noqa: E402,F401
