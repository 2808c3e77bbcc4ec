"""Host logic of the int16x2 launch planner (no GPU): csrc/plan.h is compiled on its own with
the host compiler and checked by tests/plan_check.cpp (tile choice for every query length up to
70,000, CTA task coverage and row targets, launch-bin order); every (mode, register tile) the
tile choice can produce must be one that csrc/sw16_inst.cuh instantiates, else its launch would
fail at run time."""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1908_10574_gb300", "csrc")


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"),
                 os.path.dirname(os.path.dirname(shutil.which("nvcc") or "")), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    return None


def _instantiated_tiles():
    """(mode, R) pairs of the kernel instantiations, read from the CM_R_CASES lists."""
    txt = open(os.path.join(CSRC, "sw16_inst.cuh")).read()
    out, named, mode = {}, set(), None
    for line in txt.splitlines():
        m = re.match(r"#(?:el)?if CM_MODE == (\d)", line)
        if m:
            mode = int(m.group(1))
            named.add(mode)
            continue
        if line.startswith("#else"):
            rest = {0, 1, 2, 3} - named
            assert len(rest) == 1
            mode = rest.pop()
            continue
        if line.startswith("#endif"):
            mode = None
            continue
        if mode is not None:
            out.setdefault(mode, set()).update(int(r) for r in re.findall(r"X\((\d+)\)", line))
    return {(m, r) for m, rs in out.items() for r in rs}


@pytest.mark.skipif(shutil.which("g++") is None or _cuda_include() is None,
                    reason="no host C++ compiler or CUDA headers")
def test_planner(tmp_path):
    exe = str(tmp_path / "plan_check")
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC, "-I",
                    _cuda_include(), os.path.join(HERE, "plan_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-2000:]
    assert out.stdout.rstrip().endswith("ok")
    produced = {(int(m), int(r)) for m, r in re.findall(r"tile (\d) (\d+)", out.stdout)}
    inst = _instantiated_tiles()
    assert len(inst) == 16 + 8 + 32 + 16
    assert produced <= inst, sorted(produced - inst)
    assert produced == inst, sorted(inst - produced)      # no instantiation is unreachable
