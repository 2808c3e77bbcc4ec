"""ctypes binding of libcm.so (include/cm.h).  Argument marshalling only: every step of the
path runs in the library's CUDA kernels.  There is no CPU fallback; if the library is missing
or no GPU is present, calls raise."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcm.so")

CM_OK = 0
CM_ERR_CAPACITY = -6
CM_STOPPED = 1
CM_DEVICE_PTRS = 0x1
CM_ASCII = 0x2
CM_GAP_BLAST = 0x4
CM_FORCE_INT32 = 0x8
CM_TRAIN_COMPONENTS = 0x10
CM_TRAIN_COSINE = 0x20
CM_MATRIX24 = 0x40
CM_MERGE_SEQUENTIAL = 0
CM_MERGE_PARTIAL = 1

_ERRNAMES = {-1: "CM_ERR_ARG", -2: "CM_ERR_RESIDUE", -3: "CM_ERR_OOM", -4: "CM_ERR_CUDA",
             -5: "CM_ERR_TIMEOUT", -6: "CM_ERR_CAPACITY", -7: "CM_ERR_INTERNAL"}


class CMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "CM_ERR"), code, msg))
        self.code = code


class cm_stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int64), ("cells", ctypes.c_int64),
                ("cells_padded", ctypes.c_int64), ("saturated", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("sw16_launches", ctypes.c_int64),
                ("sw16_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]


class cm_params(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("mT", ctypes.c_int32), ("mU", ctypes.c_int32),
                ("use_ranker", ctypes.c_int32), ("prune_logit", ctypes.c_float),
                ("ranker_min_pairs", ctypes.c_int32), ("merge_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class cm_result(ctypes.Structure):
    _fields_ = [("n_seqs", ctypes.c_int32), ("n_clusters", ctypes.c_int32),
                ("reps", ctypes.POINTER(ctypes.c_int32)),
                ("cl_offsets", ctypes.POINTER(ctypes.c_int64)),
                ("members", ctypes.POINTER(ctypes.c_int32)),
                ("n_pairs", ctypes.c_int64),
                ("pairs", ctypes.POINTER(ctypes.c_int32)),
                ("scores", ctypes.POINTER(ctypes.c_int32)),
                ("rep_comparisons", ctypes.c_int64), ("exchange_comparisons", ctypes.c_int64),
                ("intra_comparisons", ctypes.c_int64), ("comparisons_scored", ctypes.c_int64),
                ("cells_pairs", ctypes.c_int64), ("full_merges", ctypes.c_int64),
                ("exchanges", ctypes.c_int64), ("merges", ctypes.c_int64),
                ("rounds", ctypes.c_int64), ("gpu_batches", ctypes.c_int64),
                ("exchange_waves", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("t_rep", ctypes.c_double), ("t_cells", ctypes.c_double),
                ("t_exchange", ctypes.c_double), ("t_intra", ctypes.c_double),
                ("t_rank", ctypes.c_double), ("ranker_selected", ctypes.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libcm.so is not built; run `python -c \"import __graft_entry__ as g; "
                           "g.build()\"` (or paper_1908_10574_gb300/build.py) first")
    L = ctypes.CDLL(LIB_PATH)
    p, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "cm_create": (ctypes.c_int, [ctypes.POINTER(p), ctypes.c_int]),
        "cm_destroy": (None, [p]),
        "cm_last_error": (ctypes.c_char_p, [p]),
        "cm_set_stream": (ctypes.c_int, [p, p]),
        "cm_set_tuning": (ctypes.c_int, [p, i32, i32]),
        "cm_set_batch_limit": (ctypes.c_int, [p, ctypes.c_int64]),
        "cm_set_wait_limit": (ctypes.c_int, [p, i32]),
        "cm_get_stats": (ctypes.c_int, [p, ctypes.POINTER(cm_stats)]),
        "cm_autotune": (ctypes.c_int, [p, p, p, i32, p, i32, i32, i32, ctypes.c_char_p,
                                       ctypes.POINTER(i32), ctypes.POINTER(i32), u32]),
        "cm_reset_stats": (ctypes.c_int, [p]),
        "cm_dpx_rate": (ctypes.c_int, [p, ctypes.POINTER(ctypes.c_double)]),
        "sw_score_batch": (ctypes.c_int, [p, p, p, i32, p, i64, p, i32, i32, p, u32]),
        "sw_cells_batch": (ctypes.c_int, [p, p, p, i32, p, i64, p, i32, i32, p, u32]),
        "sw_align_batch": (ctypes.c_int, [p, p, p, i32, p, i64, p, i32, i32, p, p, p, i64,
                                          ctypes.POINTER(i64), u32]),
        "sw_allpairs": (ctypes.c_int, [p, p, p, i32, p, i32, i32, i32, i64, i64, p, p, i64,
                                       ctypes.POINTER(i64), u32]),
        "cluster_merge": (ctypes.c_int, [p, p, p, i32, p, i32, i32, ctypes.POINTER(cm_params),
                                         ctypes.POINTER(ctypes.POINTER(cm_result)), u32]),
        "greedy_cluster": (ctypes.c_int, [p, p, p, i32, p, i32, i32, ctypes.POINTER(cm_params),
                                          ctypes.POINTER(ctypes.POINTER(cm_result)), u32]),
        "cluster_merge_resume": (ctypes.c_int, [p, p, p, i32, p, i32, i32,
                                                ctypes.POINTER(cm_params), ctypes.c_char_p,
                                                ctypes.c_double,
                                                ctypes.POINTER(ctypes.POINTER(cm_result)), u32]),
        "cm_result_free": (None, [ctypes.POINTER(cm_result)]),
        "cm_ranker_num_params": (i64, []),
        "cm_ranker_init": (ctypes.c_int, [p, ctypes.c_uint64]),
        "cm_ranker_set_params": (ctypes.c_int, [p, p, i64]),
        "cm_ranker_get_params": (ctypes.c_int, [p, p, i64]),
        "cm_ranker_save": (ctypes.c_int, [p, ctypes.c_char_p]),
        "cm_ranker_load": (ctypes.c_int, [p, ctypes.c_char_p]),
        "cm_ranker_standardize": (ctypes.c_int, [p, p, p, i32, i32, u32]),
        "cm_ranker_loss_grad": (ctypes.c_int, [p, p, p, i32, p, p, i64, p, p, u32]),
        "cm_ranker_train": (ctypes.c_int, [p, p, p, i32, p, p, i64, i32, i32, ctypes.c_float,
                                           ctypes.c_uint64, p, u32]),
        "cm_ranker_embed": (ctypes.c_int, [p, p, p, i32, p, u32]),
        "cm_ranker_logits": (ctypes.c_int, [p, p, p, i32, p, i64, p, u32]),
        "sw_cells_batch_noalloc": (ctypes.c_int, [p, p, i32, p, i64, p, i32, i32, p, p, u32,
                                                  ctypes.c_char_p, i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(ctx, code):
    if code != CM_OK:
        raise CMError(code, lib().cm_last_error(ctx).decode(errors="replace"))
