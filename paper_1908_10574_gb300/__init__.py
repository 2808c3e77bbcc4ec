"""GB300-native batched Smith-Waterman scoring and ClusterMerge precise clustering.

Thin Python binding of libcm.so (see include/cm.h).  Host inputs are numpy arrays; device
inputs are torch CUDA tensors (then every array must be on the GPU and the current torch
stream is used).  Names follow the C ABI: sw_score_batch, sw_cells_batch, sw_allpairs.

The library is loaded on first use; importing the package does not need a GPU.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _lib as _L
from ._lib import (CMError, CM_ASCII, CM_GAP_BLAST, CM_FORCE_INT32, CM_DEVICE_PTRS,  # noqa: F401
                   CM_TRAIN_COMPONENTS, CM_TRAIN_COSINE, CM_MERGE_SEQUENTIAL, CM_MERGE_PARTIAL,
                   CM_MATRIX24, CM_STOPPED)

__all__ = ["Context", "sw_score_batch", "sw_cells_batch", "sw_allpairs", "CMError",
           "default_context", "sw_cells_batch_noalloc", "cluster_merge", "ops_to_cigar"]


def _is_torch_cuda(x):
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor) and x.is_cuda


def _ptr(x):
    if x is None:
        return None
    if _is_torch_cuda(x):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


class Context:
    """Owns a cm_ctx (stream, device scratch, tuning) on one CUDA device."""

    def __init__(self, device: int = 0):
        L = _L.lib()
        h = ctypes.c_void_p()
        code = L.cm_create(ctypes.byref(h), int(device))
        if code != 0:
            raise CMError(code, "cm_create failed (no usable CUDA device %d?)" % device)
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            _L.lib().cm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- plumbing -------------------------------------------------------------------------
    def _prep(self, arrays):
        dev = [_is_torch_cuda(a) for a in arrays if a is not None]
        if any(dev) and not all(dev):
            raise ValueError("mix of host and device arrays: pass all numpy or all CUDA tensors")
        if dev and dev[0]:
            import torch
            _L.check(self._h, _L.lib().cm_set_stream(
                self._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
            return CM_DEVICE_PTRS
        _L.check(self._h, _L.lib().cm_set_stream(self._h, None))
        return 0

    @staticmethod
    def _host(x, dtype, shape=None):
        a = np.asarray(x)
        if (np.dtype(dtype).kind in "iu" and a.dtype != dtype and a.size and
                a.dtype.kind in "iubf"):
            # a narrowing cast would wrap (2^32 + 5 -> 5): values must fit the C type exactly
            info = np.iinfo(dtype)
            if a.dtype.kind == "f" and not np.array_equal(a, np.round(a)):
                raise ValueError("non-integer values for a %s argument" % np.dtype(dtype).name)
            if a.min() < info.min or a.max() > info.max:
                raise ValueError("values outside the %s range" % np.dtype(dtype).name)
        x = np.ascontiguousarray(a, dtype=dtype)
        if shape is not None:
            x = x.reshape(shape)
        return x

    def _inputs(self, seqs, offsets, matrix, pairs=None):
        if _is_torch_cuda(seqs):
            import torch
            for t, dt in ((seqs, torch.uint8), (offsets, torch.int64), (matrix, torch.int8)):
                if t.dtype != dt or not t.is_contiguous():
                    raise TypeError("device inputs must be contiguous %s" % dt)
            if pairs is not None and (pairs.dtype != torch.int32 or not pairs.is_contiguous()):
                raise TypeError("device pairs must be contiguous int32")
            if matrix.numel() not in (400, 576):
                raise ValueError("matrix must have 400 (20 x 20) or 576 (24 x 24) entries")
            return seqs, offsets, matrix, pairs
        seqs = self._host(seqs, np.uint8)
        offsets = self._host(offsets, np.int64)
        matrix = self._host(matrix, np.int8, (-1,))
        if matrix.size not in (400, 576):
            raise ValueError("matrix must have 400 (20 x 20) or 576 (24 x 24) entries")
        if pairs is not None:
            pairs = self._host(pairs, np.int32, (-1, 2))
        return seqs, offsets, matrix, pairs

    @staticmethod
    def _matrix_flag(matrix):
        """CM_MATRIX24 for a 24 x 24 matrix (576 entries), else 0."""
        n = matrix.numel() if hasattr(matrix, "numel") else matrix.size
        return CM_MATRIX24 if n == 576 else 0

    def stats(self):
        s = _L.cm_stats()
        _L.check(self._h, _L.lib().cm_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def reset_stats(self):
        _L.check(self._h, _L.lib().cm_reset_stats(self._h))

    def dpx_rate(self):
        """Measured DPX max-add issue rate, lane-operations per clock per SM (cm_dpx_rate)."""
        v = ctypes.c_double(0.0)
        _L.check(self._h, _L.lib().cm_dpx_rate(self._h, ctypes.byref(v)))
        return v.value

    def autotune(self, seqs, offsets, matrix, gap_open, gap_extend, sample_seqs=0,
                 cache_path=None, flags=0):
        """Pick the CTA width and warp-stream length by timing a sample (see cm_autotune);
        returns (warps_per_cta, rows_per_warp)."""
        seqs, offsets, matrix, _ = self._inputs(seqs, offsets, matrix)
        flags |= self._prep([seqs, offsets, matrix])
        flags |= self._matrix_flag(matrix)
        w, r = ctypes.c_int32(0), ctypes.c_int32(0)
        _L.check(self._h, _L.lib().cm_autotune(
            self._h, _ptr(seqs), _ptr(offsets), int(offsets.shape[0]) - 1, _ptr(matrix),
            int(gap_open), int(gap_extend), int(sample_seqs),
            cache_path.encode() if cache_path else None, ctypes.byref(w), ctypes.byref(r), flags))
        return w.value, r.value

    def set_tuning(self, warps_per_cta=0, rows_per_warp=0):
        _L.check(self._h, _L.lib().cm_set_tuning(self._h, int(warps_per_cta), int(rows_per_warp)))

    def set_batch_limit(self, max_slots=0):
        """Pair slots of one device batch of ClusterMerge's representative wave (0: default)."""
        _L.check(self._h, _L.lib().cm_set_batch_limit(self._h, int(max_slots)))

    def set_wait_limit(self, polls=0):
        """Polls (~100 ns each) before the long-pair pipeline wait gives up with
        CM_ERR_TIMEOUT (0: the default of 2^24)."""
        _L.check(self._h, _L.lib().cm_set_wait_limit(self._h, int(polls)))

    # ---- entry points ---------------------------------------------------------------------
    def sw_score_batch(self, seqs, offsets, pairs, matrix, gap_open, gap_extend, flags=0,
                       out=None):
        seqs, offsets, matrix, pairs = self._inputs(seqs, offsets, matrix, pairs)
        flags |= self._prep([seqs, offsets, matrix, pairs])
        flags |= self._matrix_flag(matrix)
        n = int(offsets.shape[0]) - 1
        npairs = int(pairs.shape[0])
        if out is None:
            if flags & CM_DEVICE_PTRS:
                import torch
                out = torch.empty(npairs, dtype=torch.int32, device=seqs.device)
            else:
                out = np.empty(npairs, dtype=np.int32)
        _L.check(self._h, _L.lib().sw_score_batch(self._h, _ptr(seqs), _ptr(offsets), n,
                                                  _ptr(pairs), npairs, _ptr(matrix),
                                                  int(gap_open), int(gap_extend), _ptr(out),
                                                  flags))
        return out

    def sw_cells_batch(self, seqs, offsets, pairs, matrix, gap_open, gap_extend, flags=0,
                       out=None):
        seqs, offsets, matrix, pairs = self._inputs(seqs, offsets, matrix, pairs)
        flags |= self._prep([seqs, offsets, matrix, pairs])
        flags |= self._matrix_flag(matrix)
        n = int(offsets.shape[0]) - 1
        npairs = int(pairs.shape[0])
        if out is None:
            if flags & CM_DEVICE_PTRS:
                import torch
                out = torch.empty((npairs, 5), dtype=torch.int32, device=seqs.device)
            else:
                out = np.empty((npairs, 5), dtype=np.int32)
        _L.check(self._h, _L.lib().sw_cells_batch(self._h, _ptr(seqs), _ptr(offsets), n,
                                                  _ptr(pairs), npairs, _ptr(matrix),
                                                  int(gap_open), int(gap_extend), _ptr(out),
                                                  flags))
        return out

    def sw_align_batch(self, seqs, offsets, pairs, matrix, gap_open, gap_extend, flags=0):
        """One optimal local alignment per pair (see sw_align_batch in cm.h).  Host arrays
        only.  Returns (cells (n, 5) int32, offsets (n + 1,) int64, runs int32); the runs of
        pair k are runs[offsets[k]:offsets[k + 1]], each (length << 2) | op with op 0 = M,
        1 = I, 2 = D (see ops_to_cigar)."""
        seqs, offsets, matrix, pairs = self._inputs(seqs, offsets, matrix, pairs)
        flags |= self._prep([seqs, offsets, matrix, pairs])
        flags |= self._matrix_flag(matrix)
        if flags & CM_DEVICE_PTRS:
            raise TypeError("sw_align_batch takes host arrays")
        n = int(offsets.shape[0]) - 1
        npairs = int(pairs.shape[0])
        cells = np.empty((npairs, 5), dtype=np.int32)
        offs = np.empty(npairs + 1, dtype=np.int64)
        total = ctypes.c_int64(0)
        cap = 0
        for _attempt in range(2):
            runs = np.empty(max(cap, 1), dtype=np.int32)
            code = _L.lib().sw_align_batch(self._h, _ptr(seqs), _ptr(offsets), n, _ptr(pairs),
                                           npairs, _ptr(matrix), int(gap_open), int(gap_extend),
                                           _ptr(cells), _ptr(offs), _ptr(runs), cap,
                                           ctypes.byref(total), flags)
            if code == _L.CM_ERR_CAPACITY:
                cap = int(total.value)
                continue
            _L.check(self._h, code)
            return cells, offs, runs[:int(total.value)]
        raise CMError(_L.CM_ERR_CAPACITY, "capacity retry failed")

    def sw_allpairs(self, seqs, offsets, matrix, gap_open, gap_extend, T, part=0, n_parts=1,
                    flags=0, capacity=None, pairs_out=None, scores_out=None):
        """Significant pairs (i < j, f > T) of one part of the all-against-all triangle.
        Returns (pairs (k, 2) int32, scores (k,) int32)."""
        seqs, offsets, matrix, _ = self._inputs(seqs, offsets, matrix)
        flags |= self._prep([seqs, offsets, matrix])
        flags |= self._matrix_flag(matrix)
        n = int(offsets.shape[0]) - 1
        found = ctypes.c_int64(0)
        dev = bool(flags & CM_DEVICE_PTRS)
        if capacity is None:
            capacity = pairs_out.shape[0] if pairs_out is not None else 1 << 16
        for _attempt in range(2):
            if pairs_out is None or pairs_out.shape[0] < capacity:
                if dev:
                    import torch
                    pairs_out = torch.empty((capacity, 2), dtype=torch.int32, device=seqs.device)
                    scores_out = torch.empty(capacity, dtype=torch.int32, device=seqs.device)
                else:
                    pairs_out = np.empty((capacity, 2), dtype=np.int32)
                    scores_out = np.empty(capacity, dtype=np.int32)
            code = _L.lib().sw_allpairs(self._h, _ptr(seqs), _ptr(offsets), n, _ptr(matrix),
                                        int(gap_open), int(gap_extend), int(T), int(part),
                                        int(n_parts), _ptr(pairs_out), _ptr(scores_out),
                                        int(capacity), ctypes.byref(found), flags)
            if code == _L.CM_ERR_CAPACITY:
                capacity = int(found.value)
                pairs_out = scores_out = None
                continue
            _L.check(self._h, code)
            k = int(found.value)
            return pairs_out[:k], scores_out[:k]
        raise CMError(_L.CM_ERR_CAPACITY, "capacity retry failed")


    def cluster_merge(self, seqs, offsets, matrix, gap_open, gap_extend, T, mT, mU, flags=0,
                      use_ranker=False, prune_logit=0.0, ranker_min_pairs=0, merge_mode=0,
                      state_path=None, budget_seconds=0.0):
        """ClusterMerge (Algorithms 1 and 2 with the Sec. 4 transitivity test) plus the
        intra-cluster all-against-all.  Returns a dict: clusters [(rep, [members])], pairs
        (k, 3) int64 (i, j, score) sorted, and the comparison counters.  With `state_path`
        (cluster_merge_resume): resumes from the checkpoint there if there is one, and with
        budget_seconds > 0 stops at the first round boundary past the budget, saves the
        state and returns None."""
        seqs, offsets, matrix, _ = self._inputs(seqs, offsets, matrix)
        flags |= self._prep([seqs, offsets, matrix])
        flags |= self._matrix_flag(matrix)
        n = int(offsets.shape[0]) - 1
        prm = _L.cm_params(int(T), int(mT), int(mU), int(bool(use_ranker)), float(prune_logit),
                           int(ranker_min_pairs), int(merge_mode))
        res = ctypes.POINTER(_L.cm_result)()
        if state_path is None:
            _L.check(self._h, _L.lib().cluster_merge(self._h, _ptr(seqs), _ptr(offsets), n,
                                                     _ptr(matrix), int(gap_open), int(gap_extend),
                                                     ctypes.byref(prm), ctypes.byref(res), flags))
            return self._result(res)
        code = _L.lib().cluster_merge_resume(self._h, _ptr(seqs), _ptr(offsets), n, _ptr(matrix),
                                             int(gap_open), int(gap_extend), ctypes.byref(prm),
                                             os.fsencode(state_path), float(budget_seconds),
                                             ctypes.byref(res), flags)
        if code == _L.CM_STOPPED:
            return None
        _L.check(self._h, code)
        return self._result(res)

    def greedy_cluster(self, seqs, offsets, matrix, gap_open, gap_extend, T, mT, mU, flags=0):
        """Incremental greedy clustering (the paper's comparison method) plus the
        intra-cluster all-against-all; same result dict as cluster_merge."""
        seqs, offsets, matrix, _ = self._inputs(seqs, offsets, matrix)
        flags |= self._prep([seqs, offsets, matrix])
        flags |= self._matrix_flag(matrix)
        n = int(offsets.shape[0]) - 1
        prm = _L.cm_params(int(T), int(mT), int(mU), 0, 0.0, 0, 0)
        res = ctypes.POINTER(_L.cm_result)()
        _L.check(self._h, _L.lib().greedy_cluster(self._h, _ptr(seqs), _ptr(offsets), n,
                                                  _ptr(matrix), int(gap_open), int(gap_extend),
                                                  ctypes.byref(prm), ctypes.byref(res), flags))
        return self._result(res)

    @staticmethod
    def _result(res):
        try:
            R = res.contents
            nc = R.n_clusters
            off = np.ctypeslib.as_array(R.cl_offsets, shape=(nc + 1,)).copy()
            mem = (np.ctypeslib.as_array(R.members, shape=(int(off[-1]),)).copy()
                   if off[-1] > 0 else np.zeros(0, np.int32))
            reps = np.ctypeslib.as_array(R.reps, shape=(nc,)).copy() if nc else np.zeros(0, np.int32)
            k = int(R.n_pairs)
            pairs = np.zeros((k, 3), dtype=np.int64)
            if k:
                pairs[:, :2] = np.ctypeslib.as_array(R.pairs, shape=(k, 2))
                pairs[:, 2] = np.ctypeslib.as_array(R.scores, shape=(k,))
            stats = {f: getattr(R, f) for f, _ in R._fields_
                     if f not in ("reps", "cl_offsets", "members", "pairs", "scores")}
        finally:
            _L.lib().cm_result_free(res)
        clusters = [(int(reps[i]), mem[off[i]:off[i + 1]].tolist()) for i in range(nc)]
        return {"clusters": clusters, "pairs": pairs, "stats": stats}


    # ---- learned representative ranker -------------------------------------------------
    def ranker_num_params(self):
        return int(_L.lib().cm_ranker_num_params())

    def ranker_init(self, seed=1908):
        _L.check(self._h, _L.lib().cm_ranker_init(self._h, int(seed)))

    def ranker_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _L.check(self._h, _L.lib().cm_ranker_set_params(self._h, _ptr(p), len(p)))

    def ranker_get_params(self):
        out = np.empty(self.ranker_num_params(), dtype=np.float32)
        _L.check(self._h, _L.lib().cm_ranker_get_params(self._h, _ptr(out), len(out)))
        return out

    def ranker_save(self, path):
        """Write the ranker parameters to `path` (see cm_ranker_save)."""
        _L.check(self._h, _L.lib().cm_ranker_save(self._h, os.fsencode(path)))

    def ranker_load(self, path):
        """Read ranker parameters saved by ranker_save (see cm_ranker_load)."""
        _L.check(self._h, _L.lib().cm_ranker_load(self._h, os.fsencode(path)))

    def ranker_standardize(self, seqs, offsets, max_sample=1024, flags=0):
        seqs, offsets = self._host_seqs(seqs, offsets)
        self._prep([seqs])
        _L.check(self._h, _L.lib().cm_ranker_standardize(self._h, _ptr(seqs), _ptr(offsets),
                                                         len(offsets) - 1, int(max_sample), flags))

    def _host_seqs(self, seqs, offsets):
        return self._host(seqs, np.uint8), self._host(offsets, np.int64)

    def ranker_loss_grad(self, seqs, offsets, pairs, labels, flags=0):
        seqs, offsets = self._host_seqs(seqs, offsets)
        pairs = self._host(pairs, np.int32, (-1, 2))
        labels = self._host(labels, np.float32)
        self._prep([seqs])
        loss = np.zeros(1, np.float32)
        grad = np.empty(self.ranker_num_params(), np.float32)
        _L.check(self._h, _L.lib().cm_ranker_loss_grad(
            self._h, _ptr(seqs), _ptr(offsets), len(offsets) - 1, _ptr(pairs), _ptr(labels),
            len(pairs), _ptr(loss), _ptr(grad), flags))
        return float(loss[0]), grad

    def ranker_train(self, seqs, offsets, pairs, labels, epochs=1, batch_pairs=256, lr=1e-3,
                     seed=1908, flags=0):
        seqs, offsets = self._host_seqs(seqs, offsets)
        pairs = self._host(pairs, np.int32, (-1, 2))
        labels = self._host(labels, np.float32)
        self._prep([seqs])
        loss = np.zeros(1, np.float32)
        _L.check(self._h, _L.lib().cm_ranker_train(
            self._h, _ptr(seqs), _ptr(offsets), len(offsets) - 1, _ptr(pairs), _ptr(labels),
            len(pairs), int(epochs), int(batch_pairs), float(lr), int(seed), _ptr(loss), flags))
        return float(loss[0])

    def ranker_embed(self, seqs, offsets, flags=0):
        seqs, offsets = self._host_seqs(seqs, offsets)
        self._prep([seqs])
        out = np.empty((len(offsets) - 1, 128), np.float32)
        _L.check(self._h, _L.lib().cm_ranker_embed(self._h, _ptr(seqs), _ptr(offsets),
                                                   len(offsets) - 1, _ptr(out), flags))
        return out

    def ranker_logits(self, seqs, offsets, pairs, flags=0):
        seqs, offsets = self._host_seqs(seqs, offsets)
        pairs = self._host(pairs, np.int32, (-1, 2))
        self._prep([seqs])
        out = np.empty(len(pairs), np.float32)
        _L.check(self._h, _L.lib().cm_ranker_logits(self._h, _ptr(seqs), _ptr(offsets),
                                                    len(offsets) - 1, _ptr(pairs), len(pairs),
                                                    _ptr(out), flags))
        return out


_default = {}


def default_context(device: int = 0) -> Context:
    if device not in _default:
        _default[device] = Context(device)
    return _default[device]


def sw_score_batch(seqs, offsets, pairs, matrix, gap_open, gap_extend, flags=0, out=None):
    return default_context().sw_score_batch(seqs, offsets, pairs, matrix, gap_open, gap_extend,
                                            flags, out)


def sw_cells_batch(seqs, offsets, pairs, matrix, gap_open, gap_extend, flags=0, out=None):
    return default_context().sw_cells_batch(seqs, offsets, pairs, matrix, gap_open, gap_extend,
                                            flags, out)


def sw_allpairs(seqs, offsets, matrix, gap_open, gap_extend, T, part=0, n_parts=1, flags=0,
                capacity=None):
    return default_context().sw_allpairs(seqs, offsets, matrix, gap_open, gap_extend, T, part,
                                         n_parts, flags, capacity)


def ops_to_cigar(runs):
    """CIGAR text of run-length alignment ops ((length << 2) | op, op 0 = M, 1 = I, 2 = D)."""
    return "".join("%d%s" % (int(x) >> 2, "MID"[int(x) & 3]) for x in runs)


def sw_cells_batch_noalloc(seqs, offsets, pairs, matrix, gap_open, gap_extend, cells_out,
                           flags=0):
    """Allocation-free alignment cells (see include/cm.h): `seqs` (uint8), `offsets` (int64,
    n+1), `pairs` (int32, (k, 2)) and `cells_out` (int32, (k, 5), caller-allocated) are
    contiguous torch CUDA tensors on the current device; `matrix` is a host array of 400
    int8-range values; the current torch stream is used.  Nothing is allocated by the call."""
    import torch
    dev = torch.cuda.current_device()
    for name, t, dt in (("seqs", seqs, torch.uint8), ("offsets", offsets, torch.int64),
                        ("pairs", pairs, torch.int32), ("cells_out", cells_out, torch.int32)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device.index == dev):
            raise TypeError("%s must be a CUDA tensor on the current device (cuda:%d)" % (name, dev))
        if t.dtype != dt or not t.is_contiguous():
            raise TypeError("%s must be a contiguous %s tensor" % (name, dt))
    if offsets.dim() != 1 or offsets.shape[0] < 1:
        raise ValueError("offsets must have shape (n_seqs + 1,)")
    if pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must have shape (k, 2)")
    if tuple(cells_out.shape) != (pairs.shape[0], 5):
        raise ValueError("cells_out must have shape (%d, 5)" % pairs.shape[0])
    m = Context._host(matrix, np.int8, (400,))
    buf = ctypes.create_string_buffer(256)
    code = _L.lib().sw_cells_batch_noalloc(
        _ptr(seqs), _ptr(offsets), int(offsets.shape[0]) - 1, _ptr(pairs), int(pairs.shape[0]),
        ctypes.c_void_p(m.ctypes.data), int(gap_open), int(gap_extend), _ptr(cells_out),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), int(flags), buf, 256)
    if code != 0:
        raise CMError(code, buf.value.decode(errors="replace"))
    return cells_out


def cluster_merge(seqs, offsets, matrix, gap_open, gap_extend, T, mT, mU, flags=0,
                  use_ranker=False, prune_logit=0.0, ranker_min_pairs=0, merge_mode=0,
                  state_path=None, budget_seconds=0.0):
    return default_context().cluster_merge(seqs, offsets, matrix, gap_open, gap_extend, T, mT,
                                           mU, flags, use_ranker, prune_logit, ranker_min_pairs,
                                           merge_mode, state_path, budget_seconds)
