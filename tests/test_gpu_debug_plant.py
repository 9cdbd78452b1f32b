"""The range check of the COMET_DEBUG build catches a store aimed outside its buffer.

Runs only when the loaded library is the debug build (test_gpu_debug_build.py runs the GPU
suite against it in a child process); with the release library it is skipped.  debug_flags bit
3 makes the first thread of a copy step add 2^40 elements to its output offsets: the check must
skip those stores (the guard bands around the output stay intact) and report COMET_ERR_BOUNDS,
and the next call must run clean.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def comet():
    import paper_2102_06827_gb300 as c
    if "debug" not in c.version():
        pytest.skip("release library: the range checks are compiled out")
    return c


def test_planted_store_is_caught(comet):
    import torch
    from paper_2102_06827_gb300 import _lib
    e = "B[j,i] = A[i,j]"
    ext = dict(i=70, j=45)
    a = synth.tensor((70, 45), 71, 0).astype(np.float32)
    x = torch.from_numpy(np.ascontiguousarray(a.T)).cuda()   # column-major A[i,j]
    G = 4096
    full = torch.full((G + 70 * 45 * 4 + G,), 0xA5, dtype=torch.uint8, device="cuda")
    out = full[G:G + 70 * 45 * 4].view(torch.float32)
    planted = comet.Plan(e, ext, torch.float32, debug_flags=8)
    planted.contract([x], out, planted.workspace())
    with pytest.raises(_lib.CometError) as err:
        comet.sync_status()
    assert err.value.code == 13   # COMET_ERR_BOUNDS
    assert bool((full[:G] == 0xA5).all()) and bool((full[G + 70 * 45 * 4:] == 0xA5).all())
    clean = comet.Plan(e, ext, torch.float32)
    clean.contract([x], out, clean.workspace())
    comet.sync_status()
    got = np.reshape(out.cpu().numpy(), (45, 70), order="F")
    assert np.array_equal(got, a.T)
