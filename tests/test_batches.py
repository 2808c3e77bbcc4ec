"""Host logic of ClusterMerge's bounded device batches (no GPU): the splitter in
csrc/batches.h is compiled on its own with the host compiler and checked on random block
lists by tests/batches_check.cpp (coverage of the slot layout, the slot limit, cuts between
query rows only, greedy filling, and renumbering of the batches' significant slots)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1908_10574_gb300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="no host C++ compiler")
def test_batch_splitter(tmp_path):
    exe = str(tmp_path / "batches_check")
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC,
                    os.path.join(HERE, "batches_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe, "20000"], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok 20000")
