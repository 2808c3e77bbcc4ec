"""The C ABI library builds, loads, and exports every entry point that include/cm.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import paper_1908_10574_gb300 as cm
from paper_1908_10574_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                                 txt, flags=re.M):
                names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    names = _declared()
    assert {"cm_create", "sw_score_batch", "sw_allpairs", "sw_cells_batch"} <= names
    for n in names:
        assert hasattr(L, n), n


def test_no_gpu_fails_loudly_or_works():
    import torch
    if torch.cuda.is_available():
        return
    h = ctypes.c_void_p()
    assert _lib.lib().cm_create(ctypes.byref(h), 0) != 0
