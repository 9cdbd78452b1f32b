"""The GPU parity suite against the COMET_DEBUG build (libcomet_debug.so).

In that build the transpose, GEMM, gemv, batched and triples kernels test their global accesses
(the tensor-core kernels: every access outside their tensor maps) against the byte ranges of the
buffers they belong to and report COMET_ERR_BOUNDS instead of making them.  This test
builds it and runs the contraction, view, batch-label, reduction, gemv, transpose, emulated-FP64,
host-pipeline, guard-band, batched and triples-energy suites in a child process that loads it
(COMET_LIBRARY): every test there ends in comet_sync_status(), so any access outside a buffer
fails it.  The planted-store
test (test_gpu_debug_plant.py) runs there too and checks that the check fires.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["test_gpu_debug_plant.py", "test_gpu_contract.py", "test_gpu_views.py", "test_gpu_batch_labels.py",
          "test_gpu_reduce.py", "test_gpu_gemv.py", "test_gpu_transpose.py", "test_gpu_emu.py",
          "test_gpu_host.py", "test_gpu_canaries.py", "test_gpu_batched.py", "test_gpu_triples_energy.py"]


def test_gpu_suite_under_range_checks():
    from paper_2102_06827_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, COMET_LIBRARY=lib)
    probe = subprocess.run([sys.executable, "-c", "import paper_2102_06827_gb300 as c; print(c.version())"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert probe.returncode == 0 and "debug" in probe.stdout, probe.stdout + probe.stderr

    def run(files):
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                            *[os.path.join("tests", f) for f in files]],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
        return r.returncode, r.stdout + r.stderr

    rc, out = run(["test_gpu_debug_plant.py"])   # the check fires (and the test is not skipped)
    assert rc == 0 and "1 passed" in out, out[-4000:]
    rc, out = run(SUITES[1:])
    assert rc == 0, out[-4000:]
