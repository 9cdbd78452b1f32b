"""The scratch-free entry point, comet_contract_noalloc().

Some callers cannot allocate device memory when they contract (a memory budget fixed at
start-up, a plug-in whose host application owns every allocation, or simply no allocator at
hand).  For them the library keeps one fixed scratch array of its own, and this entry point
runs a plan with that array as its workspace.  The test calls it through the C ABI twice in a
row and compares both results with comet_contract() given a caller workspace, at the
tolerances the other GPU tests use.  It lives in its own file, collected last, so that a run
that stops at the first failure has already run every other test.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from helpers import empty_like_labels, from_dev, to_dev

pytestmark = pytest.mark.gpu

TOL_SPLIT = 1e-6
TOL_F64 = 1e-12


def _limit_bytes() -> int:
    """COMET_NOALLOC_MAX_BYTES as the public header defines it (one source for the test)."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "comet.h")).read()
    m = re.search(r"#define\s+COMET_NOALLOC_MAX_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", text)
    assert m, "COMET_NOALLOC_MAX_BYTES not found in include/comet.h"
    return int(m.group(1)) << int(m.group(2))


LIMIT = _limit_bytes()


@pytest.fixture(scope="module")
def comet():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2102_06827_gb300 as c
    return c


def _noalloc(comet, plan, ins, out):
    L = comet.lib()
    arr = (ctypes.c_void_p * len(ins))(*[t.data_ptr() for t in ins])
    import torch
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.comet_contract_noalloc(plan._h, arr, ctypes.c_void_p(out.data_ptr()), stream)


def _rel(x, ref):
    return float(np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300))


# Each case routes a different part of the scratch array: the split planes and scale words,
# the six emulated-FP64 planes, the FP64 chunk partials of a tensor-times-vector step, the FP32
# partials of a GEMM sliced along K, and the intermediates of a three-operand chain.
CASES = [
    ("C[m,n] = A[k,m] * B[k,n]", dict(m=300, n=520, k=700), "split_bf16", np.float32, TOL_SPLIT, {}),
    ("C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]", dict(i=6, j=5, k=7, a=24, b=20, c=19), "split_bf16",
     np.float64, TOL_SPLIT, {}),
    ("D[a,b] = A[a,i,j] * B[i,j,k,l] * C[k,l,b]", dict(a=40, b=36, i=6, j=5, k=7, l=4), "split_bf16",
     np.float32, TOL_SPLIT, {}),
    ("D[a,b] = A[a,i,j] * B[i,j,k,l] * C[k,l,b]", dict(a=40, b=36, i=6, j=5, k=7, l=4), "native",
     np.float64, TOL_F64, {}),
    ("C[m,n] = A[k,m] * B[k,n]", dict(m=200, n=150, k=300), "emu_f64", np.float64, TOL_F64, {}),
    ("y[n] = A[k,n] * x[k]", dict(n=700, k=5000), "split_bf16", np.float32, TOL_SPLIT, {}),
    ("y[n] = A[k,n] * x[k]", dict(n=700, k=5000), "native", np.float64, TOL_F64, {}),
    ("C[m,n] = A[k,m] * B[k,n]", dict(m=300, n=200, k=3001), "split_bf16", np.float32, TOL_SPLIT,
     dict(ksplit=0)),
]


@pytest.mark.parametrize("expr,ext,prec,dtype,tol,kw", CASES)
def test_noalloc_matches_contract_twice(comet, expr, ext, prec, dtype, tol, kw):
    import oracle
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    plan = comet.Plan(expr, ext, tdt, precision=prec, **kw)
    assert plan.workspace_bytes <= LIMIT
    if "ksplit" in kw:
        assert plan.info["steps"][0]["ksplit"] > 1
    if expr.startswith("y["):
        assert "gemv" in plan.info["steps"][0]["kernel"]
    _, out_labels, _, _, ops = oracle.parse(expr)
    arrays = [synth.tensor(tuple(ext[l] for l in ls), 21, t, dtype=dtype) for t, (_, ls) in enumerate(ops)]
    ins = [to_dev(a) for a in arrays]
    out_shape = tuple(ext[l] for l in out_labels)
    ref_out = empty_like_labels(out_shape, tdt)
    plan.contract(ins, ref_out, plan.workspace())
    comet.sync_status()
    ref = from_dev(ref_out).astype(np.float64)
    for _ in range(2):   # the second call sees the array as the first call left it
        out = empty_like_labels(out_shape, tdt)
        assert _noalloc(comet, plan, ins, out) == 0
        comet.sync_status()
        got = from_dev(out).astype(np.float64)
        assert _rel(got, ref) <= tol
        # the same plan, inputs and kernels with another workspace address: the same bits
        assert np.array_equal(got, ref)


def test_noalloc_refuses_plans_above_the_limit(comet):
    import torch
    plan = comet.Plan("C[m,n] = A[k,m] * B[k,n]", dict(m=4096, n=4096, k=4096), torch.float32,
                      precision="split_bf16")
    assert plan.workspace_bytes > LIMIT
    a = torch.zeros(16, device="cuda")
    status = _noalloc(comet, plan, [a, a], a)
    assert comet._lib.STATUS[status] == "COMET_ERR_WORKSPACE"


def test_noalloc_on_views(comet):
    # a plan on views (strided slices of stored tensors) through the scratch-free entry point
    import torch
    e = "C[i,j] = A[i,k] * B[k,j]"
    ext = dict(i=70, j=90, k=50)
    views = [(0, 0, 160, 3, 2), (2, 1, 200, 5, 2)]
    A = synth.tensor((160, 50), 24, 0).astype(np.float32)
    B = synth.tensor((50, 90), 24, 1).astype(np.float32)
    C0 = synth.tensor((70, 200), 24, 2).astype(np.float32)
    p = comet.Plan(e, ext, torch.float32, precision="split_bf16", views=views)
    ins = [to_dev(A, np.float32), to_dev(B, np.float32)]
    out_ref, out = to_dev(C0, np.float32), to_dev(C0, np.float32)
    p.contract(ins, out_ref, p.workspace())
    assert _noalloc(comet, p, ins, out) == 0
    comet.sync_status()
    assert torch.equal(out, out_ref)
