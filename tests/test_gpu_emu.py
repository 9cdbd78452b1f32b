"""GPU parity of the emulated-FP64 path (six bfloat16 slices on the tcgen05 tensor cores)
against the FP64 oracle: bit-exact on integer inputs, normwise relative error <= 1e-12 on
uniform inputs (the FP64 tolerance), tiles with ragged edges, chunked K, alpha and the
accumulating forms, multi-operand plans, a wide dynamic range, the full-size CCSD-like
workload on sampled outputs, and the bounded-wait fault injection."""
import numpy as np
import pytest

import oracle
import synth
from helpers import maxabs, normwise
from test_gpu_contract import EXPRS, inputs, run

pytestmark = pytest.mark.gpu

TOL = 1e-12
PREC = "emu_f64"


@pytest.fixture(scope="module")
def comet():
    import paper_2102_06827_gb300 as c
    return c


@pytest.mark.parametrize("expr,ext", EXPRS)
def test_integers_exact(comet, expr, ext):
    arrays = inputs(expr, ext, 21, kind="int", lo=-4, hi=4)
    C, p = run(comet, expr, ext, arrays, np.float64, precision=PREC)
    # steps with an operand without free labels run as tensor-times-vector steps
    assert p.info["steps"][0]["kernel"] in ("gemm_emu_bf16x6", "gemv")
    assert np.array_equal(C, oracle.einsum(expr, *arrays))


@pytest.mark.parametrize("expr,ext", EXPRS)
def test_uniform(comet, expr, ext):
    arrays = inputs(expr, ext, 22)
    C, _ = run(comet, expr, ext, arrays, np.float64, precision=PREC)
    ref = oracle.einsum(expr, *arrays)
    # componentwise scale sum |a||b| for the ill-conditioned small cases (a long dot product)
    assert maxabs(C, ref) <= TOL * float(np.max(oracle.abs_einsum(expr, *arrays)))


@pytest.mark.parametrize("M,N,K", [(128, 80, 32), (129, 81, 33), (300, 520, 100), (1, 1, 1), (1000, 7, 2000),
                                   (77, 161, 4999), (2048, 1024, 4096)])
def test_tiles_tails_and_chunks(comet, M, N, K):
    # tiles are 128 x 80 with K chunks of 192: ragged M, N and K edges, many chunks
    e = "C[m,n] = A[k,m] * B[k,n]"
    ext = dict(m=M, n=N, k=K)
    arrays = inputs(e, ext, 23)
    C, _ = run(comet, e, ext, arrays, np.float64, precision=PREC)
    if M * N * K <= 2e8:
        assert normwise(C, oracle.einsum(e, *arrays)) <= TOL
    else:
        sel = np.unique(synth.integers(23, 99, 4096, 0, M * N - 1).astype(np.int64))
        vals = oracle.einsum_sampled(e, *arrays, sel=sel)
        assert normwise(np.ravel(C, order="F")[sel], vals) <= TOL


def test_alpha_accumulate_and_chain(comet):
    e = "C[i,j] = A[i,k] * B[k,j]"
    ext = dict(i=40, j=50, k=30)
    A, B = inputs(e, ext, 24, kind="int")
    C0 = synth.tensor((40, 50), 24, 9, kind="int")
    base = oracle.einsum(e, A, B)
    C, _ = run(comet, "C[i,j] = 2.5 * A[i,k] * B[k,j]", ext, [A, B], np.float64, precision=PREC)
    assert np.array_equal(C, 2.5 * base)
    C, _ = run(comet, "C[i,j] += A[i,k] * B[k,j]", ext, [A, B], np.float64, precision=PREC, out_init=C0)
    assert np.array_equal(C, C0 + base)
    C, _ = run(comet, "C[i,j] -= A[i,k] * B[k,j]", ext, [A, B], np.float64, precision=PREC, out_init=C0)
    assert np.array_equal(C, C0 - base)
    e = "D[a,b] = A[a,i,j] * B[i,j,k,l] * C[k,l,b]"
    ext = dict(a=20, b=24, i=5, j=6, k=7, l=4)
    arrays = inputs(e, ext, 25)
    C, _ = run(comet, e, ext, arrays, np.float64, precision=PREC)
    assert normwise(C, oracle.einsum(e, *arrays)) <= TOL


def test_wide_dynamic_range(comet):
    # rows of A scaled by 2^-30 .. 2^0 and a normal B: the fixed-point slices follow the largest
    # magnitude, so the small rows keep their absolute (not relative) accuracy; the normwise
    # error stays at the FP64 tolerance
    e = "C[m,n] = A[k,m] * B[k,n]"
    M, N, K = 200, 150, 700
    A = synth.tensor((K, M), 26, 0)
    A = A * np.exp2(-np.floor(synth.uniform(26, 1, M) * 15 + 15))[None, :]
    B = synth.tensor((K, N), 26, 2, kind="normal")
    C, _ = run(comet, e, dict(m=M, n=N, k=K), [np.asfortranarray(A), B], np.float64, precision=PREC)
    assert normwise(C, oracle.einsum(e, np.asfortranarray(A), B)) <= TOL


def test_large_chunk_sums_exact(comet):
    # every slice of every element equal to 127 (x' = X 2^-46 with X = 127 (256^6 - 1) / 255 in
    # balanced base 256), some elements negated: the weight-group sums of a 192-K chunk then reach
    # 5 x 127^2 x 192 = 1.5e7, above 2^22, where the drain's full-rate conversion does not hold and
    # its exact fallback must take over; K spans three chunks and a tail
    X = 127 * (256 ** 6 - 1) // 255
    x = float(X) / 2.0 ** 46
    assert float(X) == X and 1.0 <= x < 2.0
    e = "C[m,n] = A[k,m] * B[k,n]"
    M, N, K = 130, 100, 500
    sa = np.where(synth.integers(27, 0, K * M, 0, 9) < 2, -1.0, 1.0).reshape((K, M), order="F")
    A = np.asfortranarray(x * sa)
    B = np.asfortranarray(np.full((K, N), x))
    C, _ = run(comet, e, dict(m=M, n=N, k=K), [A, B], np.float64, precision=PREC)
    ref = oracle.einsum(e, A, B)
    assert normwise(C, ref) <= TOL
    # about 80 % of the signs positive: the sums stay large (net 0.6 K of same-sign products)
    assert np.abs(ref).max() >= 0.5 * K * x * x


def test_ccsd_like_full_size_sampled(comet):
    e = "C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]"
    ext = dict(i=64, j=64, k=64, a=192, b=192, c=192)
    s = 1.0 / np.sqrt(64 * 192)
    A = synth.tensor((64, 192, 192, 64), 1, 0, scale=s)
    B = synth.tensor((192, 192, 64, 64), 2, 0, scale=s)
    sel = np.unique(synth.integers(27, 0, 20000, 0, 64 * 192 * 64 * 192 - 1).astype(np.int64))
    ref = oracle.einsum_sampled(e, A, B, sel=sel)
    C, _ = run(comet, e, ext, [A, B], np.float64, precision=PREC)
    assert normwise(np.ravel(C, order="F")[sel], ref) <= TOL


def test_timeout_surfaces_and_context_survives(comet):
    e = "C[m,n] = A[k,m] * B[k,n]"
    ext = dict(m=256, n=160, k=64)
    arrays = inputs(e, ext, 28, kind="int")
    with pytest.raises(comet.CometError) as err:
        run(comet, e, ext, arrays, np.float64, precision=PREC, debug_flags=1, timeout_ms=100)
    assert err.value.name == "COMET_ERR_TIMEOUT"
    C, _ = run(comet, e, ext, arrays, np.float64, precision=PREC)
    assert np.array_equal(C, oracle.einsum(e, *arrays))
