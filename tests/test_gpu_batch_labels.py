"""GPU parity of contractions with batch labels (a label on both inputs and the result; the
Hadamard / batched-GEMM case) against the FP64 oracle in every precision: batched GEMMs with the
batch label fastest, slowest and in the middle, pure Hadamard products, a label shared by three
operands, batched tensor-times-vector steps and a batched multi-operand chain."""
import numpy as np
import pytest

import oracle
from helpers import maxabs
from test_gpu_contract import inputs, run

pytestmark = pytest.mark.gpu

CASES = [
    ("C[b,i,j] = A[b,i,k] * B[b,k,j]", dict(b=5, i=40, j=70, k=33)),
    ("C[i,j,b] = A[i,k,b] * B[k,j,b]", dict(b=3, i=130, j=90, k=300)),
    ("C[i,b,j] = A[k,i,b] * B[j,b,k]", dict(b=4, i=20, j=30, k=50)),
    ("C[i,j] = A[i,j] * B[i,j]", dict(i=300, j=170)),
    ("s[] = x[i] * y[i] * z[i]", dict(i=5000)),
    ("y[b,r] = M[b,c,r] * x[b,c]", dict(b=6, r=300, c=700)),
    ("D[b,i] = A[b,i,j] * B[b,j,k] * C[b,k]", dict(b=4, i=30, j=20, k=25)),
]
PRECS = [("native", np.float64, 1e-12), ("split_bf16", np.float32, 1e-6), ("emu_f64", np.float64, 1e-12)]


@pytest.fixture(scope="module")
def comet():
    import paper_2102_06827_gb300 as c
    return c


@pytest.mark.parametrize("expr,ext", CASES)
@pytest.mark.parametrize("prec,dtype,tol", PRECS)
def test_batch_labels_integers_exact(comet, expr, ext, prec, dtype, tol):
    arrays = inputs(expr, ext, 41, kind="int", lo=-3, hi=3)
    C, p = run(comet, expr, ext, arrays, dtype, precision=prec)
    assert any(s["batch"] for s in p.info["steps"])
    assert np.array_equal(C, oracle.einsum(expr, *arrays))


@pytest.mark.parametrize("expr,ext", CASES)
@pytest.mark.parametrize("prec,dtype,tol", PRECS)
def test_batch_labels_uniform(comet, expr, ext, prec, dtype, tol):
    arrays = [a.astype(dtype) for a in inputs(expr, ext, 42)]
    C, _ = run(comet, expr, ext, arrays, dtype, precision=prec)
    a64 = [a.astype(np.float64) for a in arrays]
    ref = oracle.einsum(expr, *a64)
    scale = float(np.max(oracle.abs_einsum(expr, *a64)))
    # FP32 storage: the result is rounded once more to FP32
    limit = tol * scale + (np.abs(ref).max() * 2.0 ** -24 if dtype == np.float32 else 0.0)
    assert maxabs(C, ref) <= limit
