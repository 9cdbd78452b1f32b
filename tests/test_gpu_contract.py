"""GPU parity of comet_contract against the FP64 oracle.

FP64 path (tensor-core f64 MMA): normwise relative error <= 1e-12, bit-exact on small integer
inputs.  Split-BF16 path: normwise relative error <= 1e-6 on uniform inputs, bit-exact on
integer inputs whose sums stay below 2^24 (every part product and partial sum is then exact).
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import empty_like_labels, from_dev, maxabs, normwise, to_dev

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12
TOL_SPLIT = 1e-6


@pytest.fixture(scope="module")
def comet():
    import paper_2102_06827_gb300 as c
    return c


def parse_shapes(expr, ext):
    _, out_labels, _, _, ops = oracle.parse(expr)
    return [tuple(ext[l] for l in ls) for _, ls in ops], tuple(ext[l] for l in out_labels)


def run(comet, expr, ext, arrays, dtype, precision="native", out_init=None, **kw):
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    p = comet.Plan(expr, ext, tdt, precision=precision, **kw)
    ins = [to_dev(a, dtype) for a in arrays]
    _, out_shape = parse_shapes(expr, ext)
    out = to_dev(out_init, dtype) if out_init is not None else empty_like_labels(out_shape, tdt)
    ws = p.workspace()
    p.contract(ins, out, ws)
    comet.sync_status()
    return from_dev(out), p


def inputs(expr, ext, seed, kind="uniform", **kw):
    shapes, _ = parse_shapes(expr, ext)
    return [synth.tensor(s, seed, t, kind=kind, **kw) for t, s in enumerate(shapes)]


# ---- FP64 path -------------------------------------------------------------------------------

def test_extent24_fp64(comet):
    e = "C[a,b,c,d] = A[a,e,b] * B[e,d,c]"
    ext = dict(a=24, b=24, c=24, d=24, e=24)
    A, B = inputs(e, ext, 0)
    C, _ = run(comet, e, ext, [A, B], np.float64)
    ref = oracle.einsum(e, A, B)
    assert normwise(C, ref) <= TOL_F64
    ratio = maxabs(C, ref) / oracle.abs_einsum(e, A, B).max()
    assert ratio <= 24 * 2.0 ** -53 * 4


EXPRS = [
    ("C[a,b,c,d] = A[a,e,b,f] * B[d,f,c,e]", dict(a=5, b=6, c=7, d=3, e=4, f=9)),
    ("C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]", dict(i=5, j=3, k=6, a=11, b=9, c=7)),
    ("C[i,j] = A[k,i] * B[j,k]", dict(i=70, j=130, k=33)),
    ("O[i,j] = x[i] * y[j]", dict(i=17, j=65)),
    ("s[] = x[i] * y[i]", dict(i=1000)),
    ("v[r] = M[c,r] * x[c]", dict(r=67, c=129)),
    ("T[a,b,c,i,j,k] = A[d,a,b,i] * B[c,d,j,k]", dict(a=5, b=3, c=4, i=3, j=6, k=2, d=7)),
]


@pytest.mark.parametrize("expr,ext", EXPRS)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_fp64_path_integers_exact(comet, expr, ext, dtype):
    arrays = inputs(expr, ext, 1, kind="int", lo=-4, hi=4)
    C, _ = run(comet, expr, ext, arrays, dtype)
    assert np.array_equal(C, oracle.einsum(expr, *arrays))


@pytest.mark.parametrize("expr,ext", EXPRS)
def test_fp64_path_uniform(comet, expr, ext):
    arrays = inputs(expr, ext, 2)
    C, _ = run(comet, expr, ext, arrays, np.float64)
    assert normwise(C, oracle.einsum(expr, *arrays)) <= TOL_F64


def test_every_ttgt_form_gives_the_same_result(comet):
    e, ext = EXPRS[0]
    arrays = inputs(e, ext, 3, kind="int", lo=-3, hi=3)
    ref = oracle.einsum(e, *arrays)
    n = comet.Plan(e, ext, "f64").info["steps"][0]["n_forms"]
    for k in range(n):
        for prec in ("native", "split_bf16"):
            C, _ = run(comet, e, ext, arrays, np.float64 if prec == "native" else np.float32, precision=prec,
                       form=k)
            assert np.array_equal(C, ref), (k, prec)


def test_alpha_accumulate_and_copy(comet):
    e = "C[i,j] = A[i,k] * B[k,j]"
    ext = dict(i=40, j=50, k=30)
    A, B = inputs(e, ext, 4, kind="int")
    C0 = synth.tensor((40, 50), 4, 9, kind="int")
    base = oracle.einsum(e, A, B)
    for prec, dt in (("native", np.float64), ("split_bf16", np.float32)):
        C, _ = run(comet, "C[i,j] = 2.5 * A[i,k] * B[k,j]", ext, [A, B], dt, precision=prec)
        assert np.array_equal(C, 2.5 * base)
        C, _ = run(comet, "C[i,j] += A[i,k] * B[k,j]", ext, [A, B], dt, precision=prec, out_init=C0)
        assert np.array_equal(C, C0 + base)
        C, _ = run(comet, "C[i,j] -= A[i,k] * B[k,j]", ext, [A, B], dt, precision=prec, out_init=C0)
        assert np.array_equal(C, C0 - base)
    # single operand: transpose with a scale (ta.copy)
    D = synth.tensor((40, 30, 7), 4, 10)
    C, _ = run(comet, "E[k,x,i] = 2.0 * D[i,k,x]", dict(i=40, k=30, x=7), [D], np.float64)
    assert np.array_equal(C, 2.0 * oracle.transpose(D, (1, 2, 0)))
    C, _ = run(comet, "E[k,x,i] = D[i,k,x]", dict(i=40, k=30, x=7), [D], np.float64)
    assert C.tobytes(order="F") == oracle.transpose(D, (1, 2, 0)).tobytes(order="F")


def test_multi_operand_chain_orders(comet):
    e = "D[a,b] = A[a,i,j] * B[i,j,k,l] * C[k,l,b]"
    ext = dict(a=20, b=24, i=5, j=6, k=7, l=4)
    arrays = inputs(e, ext, 5, kind="int", lo=-2, hi=2)
    ref = oracle.einsum(e, *arrays)
    for order in ("planned", "natural"):
        for prec, dt in (("native", np.float64), ("split_bf16", np.float32)):
            C, p = run(comet, e, ext, arrays, dt, precision=prec, order=order)
            assert np.array_equal(C, ref), (order, prec)
    arrays = inputs(e, ext, 6)
    ref = oracle.einsum(e, *arrays)
    C, _ = run(comet, e, ext, arrays, np.float64)
    assert normwise(C, ref) <= TOL_F64
    C, _ = run(comet, e, ext, arrays, np.float32, precision="split_bf16")
    assert normwise(C, ref) <= 2 * TOL_SPLIT


# ---- split-BF16 path ---------------------------------------------------------------------------

@pytest.mark.parametrize("expr,ext", EXPRS)
def test_split_integers_exact(comet, expr, ext):
    arrays = inputs(expr, ext, 7, kind="int", lo=-4, hi=4)
    C, _ = run(comet, expr, ext, arrays, np.float32, precision="split_bf16")
    assert np.array_equal(C, oracle.einsum(expr, *arrays))


def componentwise(C, expr, arrays):
    """max |C - ref| / max sum |a||b| (the scale of the componentwise error bound)."""
    return maxabs(C, oracle.einsum(expr, *arrays)) / float(np.max(oracle.abs_einsum(expr, *arrays)))


@pytest.mark.parametrize("expr,ext", EXPRS)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_split_uniform(comet, expr, ext, dtype):
    # small contractions include ill-conditioned outputs (a 1000-term dot product with
    # cancellation), so the test bounds the error by the componentwise scale sum |a||b|
    arrays = inputs(expr, ext, 8)
    C, _ = run(comet, expr, ext, arrays, dtype, precision="split_bf16")
    assert componentwise(C, expr, arrays) <= TOL_SPLIT


@pytest.mark.parametrize("M,N,K", [(128, 256, 32), (300, 520, 100), (129, 257, 33), (1, 1, 1), (1000, 7, 2000),
                                   (2048, 1024, 4096)])
def test_split_gemm_tiles_and_tails(comet, M, N, K):
    e = "C[m,n] = A[k,m] * B[k,n]"
    ext = dict(m=M, n=N, k=K)
    arrays = inputs(e, ext, 9)
    C, _ = run(comet, e, ext, arrays, np.float32, precision="split_bf16")
    ref = oracle.einsum(e, *arrays) if M * N * K <= 2e8 else None
    if ref is None:
        sel = np.unique(synth.integers(9, 99, 4096, 0, M * N - 1).astype(np.int64))
        vals = oracle.einsum_sampled(e, *arrays, sel=sel)
        assert normwise(np.ravel(C, order="F")[sel], vals) <= TOL_SPLIT
    else:
        assert normwise(C, ref) <= TOL_SPLIT


def test_ccsd_like_full_size_sampled(comet):
    # o = 64, v = 192: C[i,a,j,b] = sum_{k,c} A[k,a,c,i] * B[c,b,k,j], inputs uniform[-1,1]/sqrt(64*192)
    e = "C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]"
    ext = dict(i=64, j=64, k=64, a=192, b=192, c=192)
    s = 1.0 / np.sqrt(64 * 192)
    sel = np.unique(synth.integers(11, 0, 20000, 0, 64 * 192 * 64 * 192 - 1).astype(np.int64))
    for prec, dt, tol in (("split_bf16", np.float32, TOL_SPLIT), ("native", np.float64, TOL_F64)):
        # each form on operands of its own storage type: FP32 uniforms for the split path,
        # genuine 53-bit FP64 uniforms (not FP32 values widened) for the FP64 path
        A = synth.tensor((64, 192, 192, 64), 1, 0, scale=s, dtype=dt)
        B = synth.tensor((192, 192, 64, 64), 2, 0, scale=s, dtype=dt)
        ref = oracle.einsum_sampled(e, A, B, sel=sel)
        C, _ = run(comet, e, ext, [A, B], dt, precision=prec)
        got = np.ravel(C, order="F")[sel]
        assert normwise(got, ref) <= tol, prec
        if dt == np.float64:
            # the products round in FP64 here, so the result is not bit-identical to the oracle
            assert normwise(got, ref) > 0.0
        del A, B, C


def test_ccsd_like_full_size_integers_exact(comet):
    # the same workload on integers in [-2, 2]: every sum stays below 2^24, so the split path's
    # exact hh chunks and fixed-point parts give the exact result at full size (sampled)
    e = "C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]"
    ext = dict(i=64, j=64, k=64, a=192, b=192, c=192)
    A = synth.tensor((64, 192, 192, 64), 13, 0, kind="int", lo=-2, hi=2, dtype=np.float32)
    B = synth.tensor((192, 192, 64, 64), 13, 1, kind="int", lo=-2, hi=2, dtype=np.float32)
    sel = np.unique(synth.integers(14, 0, 20000, 0, 64 * 192 * 64 * 192 - 1).astype(np.int64))
    ref = oracle.einsum_sampled(e, A, B, sel=sel)
    C, _ = run(comet, e, ext, [A, B], np.float32, precision="split_bf16")
    assert np.array_equal(np.ravel(C, order="F")[sel], ref)


def test_timeout_surfaces_and_context_survives(comet):
    # fault injection on the host side of the protocol: one operand load is withheld, the
    # kernel's bounded wait runs out, the status word reports it, and the GPU stays usable
    e = "C[m,n] = A[k,m] * B[k,n]"
    ext = dict(m=256, n=256, k=64)
    arrays = inputs(e, ext, 12, kind="int")
    with pytest.raises(comet.CometError) as err:
        run(comet, e, ext, arrays, np.float32, precision="split_bf16", debug_flags=1, timeout_ms=100)
    assert err.value.name == "COMET_ERR_TIMEOUT"
    C, _ = run(comet, e, ext, arrays, np.float32, precision="split_bf16")
    assert np.array_equal(C, oracle.einsum(e, *arrays))


@pytest.mark.parametrize("mt,nt,tail,slices", [(17, 9, 1, 4), (19, 12, 76, 2), (25, 8, 48, 3), (23, 10, 78, 1)])
def test_split_stream_k_tail(comet, mt, nt, tail, slices):
    # whole-K tiles in full waves over 152 SMs, the partial last wave in K slices (stream-K
    # tail, up to half the SMs): ragged M and N so that tail tiles hold edges; integers stay
    # exact through the slices' FP32 partials and the reduce, alpha and += included
    e = "C[m,n] = A[m,k] * B[k,n]"
    ext = dict(m=128 * mt - 5, n=256 * nt - 7, k=300)
    p = comet.Plan(e, ext, "f32", precision="split_bf16")
    st = p.info["steps"][0]
    assert (st["ksplit"], st["tail_tiles"], st["tail_slices"]) == (1, tail if slices > 1 else 0, slices)
    arrays = inputs(e, ext, 15)
    C, _ = run(comet, e, ext, arrays, np.float32, precision="split_bf16")
    assert normwise(C, oracle.einsum(e, *arrays)) <= TOL_SPLIT
    ints = inputs(e, ext, 16, kind="int", lo=-2, hi=2)
    C0 = synth.tensor((ext["m"], ext["n"]), 16, 7, kind="int")
    C, _ = run(comet, "C[m,n] += 2.0 * A[m,k] * B[k,n]", ext, ints, np.float32, precision="split_bf16",
               out_init=C0)
    assert np.array_equal(C, C0 + 2.0 * oracle.einsum(e, *ints))


@pytest.mark.parametrize("ksplit", [0, 3, 16])
def test_split_k_slices(comet, ksplit):
    # a GEMM with few output tiles: K sliced over more work items, FP32 partials summed by a
    # second kernel (0 = the planner's choice); alpha and += go through the reduce kernel
    e = "C[m,n] = A[k,m] * B[k,n]"
    ext = dict(m=300, n=200, k=3001)
    arrays = inputs(e, ext, 13)
    ref = oracle.einsum(e, *arrays)
    C, p = run(comet, e, ext, arrays, np.float32, precision="split_bf16", ksplit=ksplit)
    assert p.info["steps"][0]["ksplit"] > 1
    assert normwise(C, ref) <= TOL_SPLIT
    ints = inputs(e, ext, 14, kind="int", lo=-2, hi=2)
    C0 = synth.tensor((300, 200), 14, 7, kind="int")
    C, _ = run(comet, "C[m,n] += 2.0 * A[k,m] * B[k,n]", ext, ints, np.float32, precision="split_bf16",
               ksplit=ksplit, out_init=C0)
    assert np.array_equal(C, C0 + 2.0 * oracle.einsum(e, *ints))
