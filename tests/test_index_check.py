"""Runs the CPU replays of kernel index arithmetic: tests/index_check.cpp (the transpose
engine's loop nests and the GEMM offset groups: bounds, vector alignment, each output written
once from the right input) and tests/batched_check.cpp (the tensor-core batched kernel: plane
rows, TMA boxes, shared and tensor memory, output offsets)."""
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


def test_batched_tc_index_arithmetic_replay(tmp_path):
    exe = str(tmp_path / "batched_check")
    csrc = os.path.join(ROOT, "paper_2102_06827_gb300", "csrc")
    src = [os.path.join(ROOT, "tests", "batched_check.cpp"), os.path.join(csrc, "plan.cpp"),
           os.path.join(csrc, "batched_plan.cpp")]
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc,
                        "-o", exe] + src, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 failures" in r.stdout


def test_triples_index_arithmetic_replay(tmp_path):
    # the fused triples kernels' staging, shared loads, element-to-entry mapping and eps reads,
    # on the workload's nine terms, for the largest block of the 4096-block table, the largest
    # of the 64 blocks the FP64 leg runs, a small ragged block, a block of extent 1 everywhere
    # and one with every remainder mod 4 and a summed label of two FP32 passes
    import numpy as np
    import synth
    from triples_terms import LABELS, SIGNS, terms
    exe = str(tmp_path / "triples_check")
    csrc = os.path.join(ROOT, "paper_2102_06827_gb300", "csrc")
    src = [os.path.join(ROOT, "tests", "triples_check.cpp"), os.path.join(csrc, "plan.cpp"),
           os.path.join(csrc, "triples_plan.cpp")]
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-o", exe] + src,
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    ext = synth.triples_blocks(4096)
    size = np.prod(ext[:, :6], axis=1)
    rows = [ext[int(np.argmax(size))], ext[int(np.argmax(size[:64]))], np.array([6, 5, 7, 4, 6, 5, 9]),
            np.ones(7, dtype=np.int64), np.array([9, 10, 11, 13, 2, 3, 40])]
    tl = terms()
    for row in rows:
        args = [exe, str(len(tl))] + tl + LABELS + [str(s) for s in SIGNS] + [str(int(x)) for x in row]
        r = subprocess.run(args, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stdout + r.stderr
        assert "0 failures" in r.stdout
