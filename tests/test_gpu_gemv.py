"""GPU parity of the tensor-times-vector steps (one operand without free labels) against the
FP64 oracle, in every precision: both thread layouts (the large operand contiguous along a free
label or along a contracted one), K chunks with a ragged tail, alpha and the accumulating forms,
a long dot product, and the two GEMV steps of a Table 1 expression."""
import numpy as np
import pytest

import oracle
import synth
from helpers import maxabs, normwise
from test_gpu_contract import inputs, run

pytestmark = pytest.mark.gpu

CASES = [
    # (expression, extents): the large operand's stride-1 label is contracted / free
    ("y[r] = M[c,r] * x[c]", dict(r=3000, c=2500)),
    ("y[r] = M[r,c] * x[c]", dict(r=3000, c=2500)),
    ("Y[d,n] = A[c,d,m,n] * C[m,c]", dict(c=40, d=30, m=20, n=25)),
    ("Y[a,i] = B[i,n,a,d] * V[d,n]", dict(i=20, n=30, a=40, d=25)),
    ("Y[m,n] = A[m,k,n] * v[k]", dict(m=7, n=300, k=1100)),
]
PRECS = [("native", np.float64, 1e-12), ("split_bf16", np.float32, 1e-6), ("emu_f64", np.float64, 1e-12)]


@pytest.fixture(scope="module")
def comet():
    import paper_2102_06827_gb300 as c
    return c


@pytest.mark.parametrize("expr,ext", CASES)
@pytest.mark.parametrize("prec,dtype,tol", PRECS)
def test_gemv_steps(comet, expr, ext, prec, dtype, tol):
    arrays = inputs(expr, ext, 31)
    C, p = run(comet, expr, ext, [a.astype(dtype) for a in arrays], dtype, precision=prec)
    assert [s["kernel"] for s in p.info["steps"]] == ["gemv"]
    ref = oracle.einsum(expr, *[a.astype(dtype).astype(np.float64) for a in arrays])
    scale = float(np.max(oracle.abs_einsum(expr, *[a.astype(dtype).astype(np.float64) for a in arrays])))
    assert maxabs(C, ref) <= tol * scale


@pytest.mark.parametrize("prec,dtype", [("native", np.float64), ("split_bf16", np.float32)])
def test_integers_exact_alpha_and_accumulate(comet, prec, dtype):
    e = "y[r] = M[c,r] * x[c]"
    ext = dict(r=513, c=2049)
    M, x = inputs(e, ext, 32, kind="int", lo=-4, hi=4)
    base = oracle.einsum(e, M, x)
    y0 = synth.tensor((513,), 32, 7, kind="int")
    C, _ = run(comet, "y[r] = 0.5 * M[c,r] * x[c]", ext, [M, x], dtype, precision=prec)
    assert np.array_equal(C, 0.5 * base)
    C, _ = run(comet, "y[r] += M[c,r] * x[c]", ext, [M, x], dtype, precision=prec, out_init=y0)
    assert np.array_equal(C, y0 + base)
    C, _ = run(comet, "y[r] -= M[c,r] * x[c]", ext, [M, x], dtype, precision=prec, out_init=y0)
    assert np.array_equal(C, y0 - base)


def test_long_dot_product(comet):
    e = "s[] = x[i] * y[i]"
    ext = dict(i=1_000_003)
    arrays = inputs(e, ext, 33)
    for prec, dt in (("native", np.float64), ("split_bf16", np.float32)):
        arr = [a.astype(dt) for a in arrays]
        C, _ = run(comet, e, ext, arr, dt, precision=prec)
        ref = oracle.einsum(e, *[a.astype(np.float64) for a in arr])
        tol = 1e-12 * float(oracle.abs_einsum(e, *[a.astype(np.float64) for a in arr]))
        if dt == np.float32:   # Dot2 is accurate far beyond FP32; the stored result is rounded once
            tol += abs(float(ref)) * 2.0 ** -24
        assert abs(float(C) - float(ref)) <= tol, prec


def test_table1_row1_two_gemv_steps(comet):
    e = "X[i,a] = A[c,d,m,n] * B[i,n,a,d] * C[m,c]"
    ext = dict(c=48, d=48, m=16, n=16, i=16, a=48)
    arrays = inputs(e, ext, 34)
    ref = oracle.einsum(e, *arrays)
    for prec, dt, tol in PRECS:
        C, p = run(comet, e, ext, [a.astype(dt) for a in arrays], dt, precision=prec)
        assert [s["kernel"] for s in p.info["steps"]] == ["gemv", "gemv"]
        assert normwise(C, ref) <= tol, prec
