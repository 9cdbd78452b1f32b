"""GPU parity of labels summed inside a single operand (reduction steps, then the rest of the
plan) against the FP64 oracle in every precision."""
import numpy as np
import pytest

import oracle
import synth
from helpers import maxabs
from test_gpu_contract import inputs, run

pytestmark = pytest.mark.gpu

CASES = [
    ("C[i] = A[i,k]", dict(i=300, k=2500)),
    ("C[k] = A[i,k]", dict(i=2500, k=300)),
    ("s[] = A[i,j]", dict(i=700, j=900)),
    ("C[a,b] = A[a,x,b,y]", dict(a=20, x=30, b=25, y=7)),
    ("C[i,j] = A[i,k,l] * B[k,j]", dict(i=40, j=50, k=30, l=9)),
    ("C[i] = A[i] * B[k]", dict(i=500, k=3000)),
]
PRECS = [("native", np.float64, 1e-12), ("split_bf16", np.float32, 1e-6), ("emu_f64", np.float64, 1e-12)]


@pytest.fixture(scope="module")
def comet():
    import paper_2102_06827_gb300 as c
    return c


@pytest.mark.parametrize("expr,ext", CASES)
@pytest.mark.parametrize("prec,dtype,tol", PRECS)
def test_private_labels(comet, expr, ext, prec, dtype, tol):
    ints = inputs(expr, ext, 51, kind="int", lo=-3, hi=3)
    C, p = run(comet, expr, ext, ints, dtype, precision=prec)
    assert p.info["steps"][0]["kernel"] == "reduce"
    assert np.array_equal(C, oracle.einsum(expr, *ints))
    arrays = [a.astype(dtype) for a in inputs(expr, ext, 52)]
    C, _ = run(comet, expr, ext, arrays, dtype, precision=prec)
    a64 = [a.astype(np.float64) for a in arrays]
    ref = oracle.einsum(expr, *a64)
    scale = float(np.max(oracle.abs_einsum(expr, *a64)))
    limit = tol * scale + (np.abs(ref).max() * 2.0 ** -24 if dtype == np.float32 else 0.0)
    assert maxabs(C, ref) <= limit


def test_reduction_alpha_and_accumulate(comet):
    e = "C[i] = A[i,k]"
    ext = dict(i=100, k=3000)
    (A,) = inputs(e, ext, 53, kind="int")
    C0 = synth.tensor((100,), 53, 5, kind="int")
    base = oracle.einsum(e, A)
    for prec, dt in (("native", np.float64), ("split_bf16", np.float32)):
        C, _ = run(comet, "C[i] = 0.25 * A[i,k]", ext, [A], dt, precision=prec)
        assert np.array_equal(C, 0.25 * base)
        C, _ = run(comet, "C[i] += A[i,k]", ext, [A], dt, precision=prec, out_init=C0)
        assert np.array_equal(C, C0 + base)
