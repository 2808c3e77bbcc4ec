"""Host logic of the ranker's training batches (no GPU): the planner in
csrc/train_batches.h is compiled on its own with the host compiler and checked on random pair
graphs by tests/train_batches_check.cpp (components against a breadth-first search, every pair
once per epoch, the batch size bound, whole components per batch, greedy filling)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1908_10574_gb300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="no host C++ compiler")
def test_train_batch_planner(tmp_path):
    exe = str(tmp_path / "train_batches_check")
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC,
                    os.path.join(HERE, "train_batches_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe, "5000"], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok 5000")
