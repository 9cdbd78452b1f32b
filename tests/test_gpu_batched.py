"""GPU parity of the batched triples path (one persistent launch over many uneven blocks)
against the oracle: stored blocks elementwise, reduced blocks through s_b = sum T*W and
q_b = sum T^2; every tile configuration, both accumulator layouts of the tensor-core split
kernel (one accumulator for K <= 32, the hh products apart when some K > 32); the full-size
workload on its smallest, middle and largest blocks; a withheld load (bounded waits);
CUDA-graph replay; the autotuner.  Split tolerance 1e-6 (normwise per block, and relative on
q_b), FP64 1e-12."""
import numpy as np
import pytest

import oracle
import synth
from batched_data import EXPR, LABELS, Blocks, shapes

pytestmark = pytest.mark.gpu

KEY = 0x5EED


@pytest.fixture(scope="module")
def comet():
    import paper_2102_06827_gb300 as c
    return c


def _store(comet, plan, blocks, pick):
    """materialise the picked blocks (store mode), other blocks skipped"""
    import torch
    outs = {}
    ptrs = [0] * blocks.n
    for b in pick:
        n = int(np.prod(shapes(blocks.ext[b])[2]))
        outs[b] = torch.zeros(n, dtype=blocks.tdt, device="cuda")
        ptrs[b] = outs[b].data_ptr()
    table = torch.tensor(ptrs, dtype=torch.int64, device="cuda")
    ws = plan.workspace()
    plan.prepare(ws)
    plan.contract(blocks.ptrs, table, ws, mode=1)
    comet.sync_status()
    return {b: np.asfortranarray(t.cpu().numpy().astype(np.float64).reshape(shapes(blocks.ext[b])[2], order="F"))
            for b, t in outs.items()}


def _reduce(comet, plan, blocks, ws=None):
    import torch
    res = torch.zeros(2 * blocks.n, dtype=torch.float64, device="cuda")
    if ws is None:
        ws = plan.workspace()
        plan.prepare(ws)
    plan.contract(blocks.ptrs, res, ws, mode=0, key=KEY)
    comet.sync_status()
    return res.cpu().numpy().reshape(-1, 2)


def _check_reduce(blocks, got, b, tol):
    A = blocks.host_operand(b, 0).astype(np.float64)
    B = blocks.host_operand(b, 1).astype(np.float64)
    s, q = oracle.triples_reduce(A, B, KEY, b)
    n = int(np.prod(shapes(blocks.ext[b])[2]))
    assert abs(got[b, 1] - q) <= tol * q, (b, got[b, 1], q)
    assert abs(got[b, 0] - s) <= tol * np.sqrt(q * n), (b, got[b, 0], s)


# uneven blocks: degenerate extents, K from 1 to 40 (K > 32 streams the B chunks and keeps the
# hh products in an accumulator of their own), strips with ragged column tails, M below 128
SMALL = np.array([[2, 3, 1, 4, 2, 3, 5], [7, 1, 2, 3, 5, 2, 1], [3, 3, 3, 3, 3, 3, 3], [1, 1, 1, 1, 1, 1, 1],
                  [9, 8, 7, 6, 5, 4, 33], [5, 6, 2, 7, 3, 4, 40], [16, 5, 9, 2, 3, 11, 6], [4, 4, 4, 8, 8, 8, 2],
                  [20, 13, 11, 3, 17, 2, 16], [1, 2, 31, 1, 9, 1, 17]])
# the same blocks with K <= 32: the tile's correction and hh products share one accumulator
SMALL_K32 = np.concatenate([SMALL[:, :6], np.minimum(SMALL[:, 6:], 32)], axis=1)


@pytest.mark.parametrize("table", ["k_to_40", "k_to_32"])
@pytest.mark.parametrize("prec,dtype,tol", [("native", np.float64, 1e-12), ("native", np.float32, 1e-12),
                                            ("split_bf16", np.float32, 1e-6), ("split_bf16", np.float64, 1e-6)])
def test_small_uneven_blocks_every_tile(comet, prec, dtype, tol, table):
    ext = SMALL if table == "k_to_40" else SMALL_K32
    if prec == "native" and table == "k_to_32":
        pytest.skip("the FP64 kernel has one accumulator layout")
    blocks = Blocks(ext, dtype, exact_blocks=range(len(ext)))
    plan = comet.BatchedPlan(EXPR, LABELS, ext, "f32" if dtype == np.float32 else "f64", precision=prec)
    if prec == "split_bf16":
        assert plan.describe()["kernel"] == "tcgen05"
        assert plan.describe()["dual_accumulators"] == (1 if table == "k_to_40" else 0)
    for cfg in range(plan.num_tiles()):
        plan.set_tile(cfg)
        outs = _store(comet, plan, blocks, range(len(ext)))
        for b, T in outs.items():
            A = blocks.host_operand(b, 0).astype(np.float64)
            B = blocks.host_operand(b, 1).astype(np.float64)
            ref = oracle.einsum(EXPR, A, B)
            err = np.abs(T - ref).max() / max(np.abs(ref).max(), 1e-300)
            # an FP32 output of the FP64 path adds its own rounding (2^-24)
            limit = 2.0 ** -23 if (prec == "native" and dtype == np.float32) else tol
            assert err <= limit, (cfg, b, err)
        got = _reduce(comet, plan, blocks)
        for b in range(len(ext)):
            _check_reduce(blocks, got, b, tol)


def test_full_size_triples_sampled(comet):
    # 4096 blocks, every extent uniform in 8..32, normal(0, 0.1); the two smallest, the
    # quartiles and the two largest blocks checked against the oracle, the largest one also
    # stored and compared element by element
    import torch
    ext = synth.triples_blocks(4096)
    fl = 2.0 * np.prod(ext, axis=1)
    order = np.argsort(fl, kind="stable")
    n = len(order)
    pick = sorted({int(order[0]), int(order[1]), int(order[n // 4]), int(order[n // 2]), int(order[3 * n // 4]),
                   int(order[-2]), int(order[-1])})
    largest = int(order[-1])
    for prec, dtype, dt, tol in (("split_bf16", np.float32, "f32", 1e-6), ("native", np.float64, "f64", 1e-12)):
        blocks = Blocks(ext, dtype, exact_blocks=pick)
        plan = comet.BatchedPlan(EXPR, LABELS, ext, dt, precision=prec)
        got = _reduce(comet, plan, blocks)
        assert np.all(got[:, 1] > 0)
        for b in pick:
            _check_reduce(blocks, got, b, tol)
        if prec == "split_bf16":
            T = _store(comet, plan, blocks, [largest])[largest]
            A = blocks.host_operand(largest, 0).astype(np.float64)
            B = blocks.host_operand(largest, 1).astype(np.float64)
            ref = oracle.einsum(EXPR, A, B)
            assert np.abs(T - ref).max() / np.abs(ref).max() <= tol
            del T, ref
        del blocks
        torch.cuda.empty_cache()


def test_withheld_load_times_out_and_context_survives(comet):
    # fault injection on the host side of the protocol: one operand load of the tensor-core
    # kernel is withheld, its bounded wait runs out, the status word reports it, and the next
    # launch on the same context is correct
    blocks = Blocks(SMALL_K32, np.float32, exact_blocks=range(len(SMALL_K32)))
    bad = comet.BatchedPlan(EXPR, LABELS, SMALL_K32, "f32", precision="split_bf16", timeout_ms=100, debug_flags=1)
    import torch
    res = torch.zeros(2 * blocks.n, dtype=torch.float64, device="cuda")
    ws = bad.workspace()
    bad.prepare(ws)
    bad.contract(blocks.ptrs, res, ws, mode=0, key=KEY)
    with pytest.raises(comet.CometError) as err:
        comet.sync_status()
    assert err.value.name == "COMET_ERR_TIMEOUT"
    good = comet.BatchedPlan(EXPR, LABELS, SMALL_K32, "f32", precision="split_bf16")
    got = _reduce(comet, good, blocks)
    for b in range(len(SMALL_K32)):
        _check_reduce(blocks, got, b, 1e-6)


def test_graph_replay_and_autotune(comet):
    import torch
    ext = synth.triples_blocks(256, 4, 16, seed=9)
    blocks = Blocks(ext, np.float32, exact_blocks=[0, 1])
    plan = comet.BatchedPlan(EXPR, LABELS, ext, "f32", precision="split_bf16")
    ws = plan.workspace()
    plan.prepare(ws)
    res = torch.zeros(2 * blocks.n, dtype=torch.float64, device="cuda")
    ms, best = plan.autotune(blocks.ptrs, res, ws, sample_blocks=64)
    assert len(ms) == plan.num_tiles() and all(m > 0 for m in ms)
    assert plan.describe()["tile_cfg"] == best == int(np.argmin(ms))
    ref = _reduce(comet, plan, blocks, ws)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    res2 = torch.zeros_like(res)
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        plan.contract(blocks.ptrs, res2, ws, mode=0, key=KEY, stream=s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        got = res2.cpu().numpy().reshape(-1, 2)
        # same kernel, same inputs: equal up to the order of the atomic additions
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-14)
    comet.sync_status()
    # a second plan of the same problem class picks up the autotuned configuration
    plan2 = comet.BatchedPlan(EXPR, LABELS, ext, "f32", precision="split_bf16")
    assert plan2.describe()["tile_cfg"] == best


# other output orders and operand layouts: the planner swaps the GEMM roles for the first two
# (the M operand is then B), which also swaps which weight factor belongs to the tile rows
LAYOUTS = ["T[c,j,k,a,b,i] = A[d,a,b,i] * B[c,d,j,k]", "T[j,c,k,i,b,a] = A[d,a,b,i] * B[c,d,j,k]",
           "T[a,c,i,j,b,k] = A[a,b,i,d] * B[d,c,j,k]"]


def _weights(expr, ext_row, key, block):
    """W over T's elements from its definition: h(key, b, oA) h(~key, b, oB), oA (oB) the part of
    the column-major offset that the first (second) operand's labels contribute."""
    _, out_labels, _, _, ops = oracle.parse(expr)
    ext = dict(zip(LABELS, [int(x) for x in ext_row]))
    shape = tuple(ext[l] for l in out_labels)
    idx = np.indices(shape)
    stride, st = {}, 1
    for l in out_labels:
        stride[l] = st
        st *= ext[l]
    a_labels = set(ops[0][1])
    oA = sum(idx[q] * stride[l] for q, l in enumerate(out_labels) if l in a_labels)
    oB = sum(idx[q] * stride[l] for q, l in enumerate(out_labels) if l not in a_labels)
    fa = np.vectorize(lambda x: oracle.triples_factor(key, block, int(x)))(oA)
    fb = np.vectorize(lambda x: oracle.triples_factor(key ^ 0xFFFFFFFF, block, int(x)))(oB)
    return fa * fb


@pytest.mark.parametrize("expr", LAYOUTS)
@pytest.mark.parametrize("prec,dtype,tol", [("split_bf16", np.float32, 1e-6), ("native", np.float64, 1e-12)])
def test_other_layouts_reduce_and_store(comet, expr, prec, dtype, tol):
    import torch
    ext = np.array([[5, 6, 3, 4, 7, 2, 9], [9, 2, 7, 3, 5, 4, 20], [4, 4, 4, 4, 4, 4, 33], [7, 3, 5, 2, 6, 8, 16]])
    _, out_labels, _, _, ops = oracle.parse(expr)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    host, dev = [], []
    for b, row in enumerate(ext):
        e = dict(zip(LABELS, [int(x) for x in row]))
        pair = [synth.tensor(tuple(e[l] for l in ls), 31, 2 * b + t, kind="normal", scale=0.1, dtype=dtype)
                for t, (_, ls) in enumerate(ops)]
        host.append(pair)
        dev.append([torch.from_numpy(np.ascontiguousarray(np.ravel(x, order="F"))).cuda() for x in pair])
    ptrs = torch.tensor([t.data_ptr() for pair in dev for t in pair], dtype=torch.int64, device="cuda")
    plan = comet.BatchedPlan(expr, LABELS, ext, "f32" if dtype == np.float32 else "f64", precision=prec)
    assert plan.describe()["swap"] == (0 if expr.startswith("T[a,c") else 1)
    for cfg in range(plan.num_tiles()):
        plan.set_tile(cfg)
        ws = plan.workspace()
        plan.prepare(ws)
        res = torch.zeros(2 * len(ext), dtype=torch.float64, device="cuda")
        plan.contract(ptrs, res, ws, mode=0, key=KEY)
        comet.sync_status()
        got = res.cpu().numpy().reshape(-1, 2)
        outs = [torch.zeros(int(np.prod([dict(zip(LABELS, row))[l] for l in out_labels])), dtype=tdt, device="cuda")
                for row in ext]
        table = torch.tensor([t.data_ptr() for t in outs], dtype=torch.int64, device="cuda")
        plan.contract(ptrs, table, ws, mode=1)
        comet.sync_status()
        for b, row in enumerate(ext):
            ref = oracle.einsum(expr, *[x.astype(np.float64) for x in host[b]])
            T = np.reshape(outs[b].cpu().numpy().astype(np.float64), ref.shape, order="F")
            assert np.abs(T - ref).max() <= tol * np.abs(ref).max(), (cfg, b)
            q = float(np.sum(ref * ref))
            s = float(np.sum(ref * _weights(expr, row, KEY, b)))
            assert abs(got[b, 1] - q) <= tol * q, (cfg, b)
            assert abs(got[b, 0] - s) <= tol * np.sqrt(q * ref.size), (cfg, b, got[b, 0], s)
