"""Runs tests/index_check.cpp: a CPU replay of the transpose engine's loop nests and of the
GEMM offset groups (bounds, vector alignment, each output written once from the right input)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_kernel_index_arithmetic_replay(tmp_path):
    exe = str(tmp_path / "index_check")
    src = [os.path.join(ROOT, "tests", "index_check.cpp"),
           os.path.join(ROOT, "paper_2102_06827_gb300", "csrc", "plan.cpp")]
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-o", exe] + src,
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 failures" in r.stdout
