"""CUDA-graph capture of the device entry points: a captured comet_contract / comet_triples_energy
replays to the same bits as the eager call, and follows new input values written into the
captured buffers.  Covers a one-step split plan, a multi-step chain with a reduction step and a
batch label, a plan on views, the emulated-FP64 form, and the fused triples energy."""
import numpy as np
import pytest

import oracle
import synth
from helpers import from_dev, normwise, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def comet():
    import paper_2102_06827_gb300 as c
    return c


def capture_and_compare(comet, plan, ins, out_shape, tdt, refill):
    import torch
    ws = plan.workspace()
    out_eager = torch.zeros(out_shape, dtype=tdt, device="cuda")
    plan.contract(ins, out_eager, ws)
    comet.sync_status()
    out_g = torch.zeros(out_shape, dtype=tdt, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.contract(ins, out_g, ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    comet.sync_status()
    assert torch.equal(out_g, out_eager)
    # new values in the captured input buffers: the replay follows them
    refill()
    plan.contract(ins, out_eager, ws)
    comet.sync_status()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out_g, out_eager)
    return from_dev(out_g)


EXPRS = [
    ("C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]", dict(i=12, j=10, k=8, a=40, b=36, c=24), "split_bf16", np.float32),
    ("D[i,l,b] = A[i,j,x,b] * B[j,k] * C[k,l,b]", dict(i=40, j=36, k=44, l=28, x=5, b=3), "split_bf16", np.float32),
    ("D[i,l] = A[i,j] * B[j,k] * C[k,l]", dict(i=64, j=48, k=80, l=40), "emu_f64", np.float64),
    ("C[i,j] = A[i,k] * B[k,j]", dict(i=96, j=80, k=72), "native", np.float64),
]


@pytest.mark.parametrize("expr,ext,prec,dtype", EXPRS)
def test_graph_replay_matches_eager(comet, expr, ext, prec, dtype):
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    _, out_labels, _, _, ops = oracle.parse(expr)
    arrays = [synth.tensor(tuple(ext[l] for l in ls), 41, t) for t, (_, ls) in enumerate(ops)]
    ins = [to_dev(a, dtype) for a in arrays]
    plan = comet.Plan(expr, ext, tdt, precision=prec)
    out_shape = tuple(reversed([ext[l] for l in out_labels]))
    fresh = [synth.tensor(tuple(ext[l] for l in ls), 42, t) for t, (_, ls) in enumerate(ops)]

    def refill():
        for t, a in zip(ins, fresh):
            t.copy_(to_dev(a, dtype))
    C = capture_and_compare(comet, plan, ins, out_shape, tdt, refill)
    # each step of a split chain adds at most the one-step bound (as in the chain tests)
    tol = 1e-6 * len(plan.info["steps"]) if prec == "split_bf16" else 1e-12
    seen = [a.astype(dtype).astype(np.float64) for a in fresh]   # the values the GPU holds
    assert normwise(C, oracle.einsum(expr, *[np.asfortranarray(a) for a in seen])) <= tol


def test_graph_replay_on_views(comet):
    import torch
    e = "C[i,j] = A[i,k] * B[k,j]"
    ext = dict(i=70, j=90, k=50)
    views = [(0, 0, 160, 3, 2), (2, 1, 200, 5, 2)]
    A = synth.tensor((160, 50), 43, 0)
    B = synth.tensor((50, 90), 43, 1)
    plan = comet.Plan(e, ext, torch.float32, precision="split_bf16", views=views)
    ins = [to_dev(A, np.float32), to_dev(B, np.float32)]
    A2 = synth.tensor((160, 50), 44, 0)

    def refill():
        ins[0].copy_(to_dev(A2, np.float32))
    C = capture_and_compare(comet, plan, ins, (200, 70), torch.float32, refill)
    got = C[:, 5:5 + 89 * 2 + 1:2]
    ref = oracle.einsum(e, np.asfortranarray(A2.astype(np.float32).astype(np.float64)[3:3 + 69 * 2 + 1:2, :]),
                        B.astype(np.float32).astype(np.float64))
    assert normwise(got, ref) <= 1e-6


def test_graph_replay_triples_energy(comet):
    import torch
    from triples_terms import LABELS, SIGNS, block_inputs, terms
    exts = [dict(a=6, b=5, c=7, i=4, j=6, k=5, d=9), dict(a=9, b=4, c=5, i=7, j=3, k=6, d=12)]
    plan = comet.TriplesPlan(terms(), LABELS, [[e[l] for l in LABELS] for e in exts], SIGNS, torch.float64)
    keep, optr, eptr = [], [], []
    for b, e in enumerate(exts):
        ops, eps = block_inputs(e, 45, b)
        for pair in ops:
            for x in pair:
                t = torch.from_numpy(np.ascontiguousarray(np.ravel(x, order="F"))).cuda()
                keep.append(t)
                optr.append(t.data_ptr())
        for x in eps:
            t = torch.from_numpy(np.asarray(x)).cuda()
            keep.append(t)
            eptr.append(t.data_ptr())
    opt = torch.tensor(optr, dtype=torch.int64, device="cuda")
    ept = torch.tensor(eptr, dtype=torch.int64, device="cuda")
    ws = plan.workspace()
    plan.prepare(ws)
    en_eager = torch.empty(2, dtype=torch.float64, device="cuda")
    plan.energy(opt, ept, en_eager, ws)
    comet.sync_status()
    en_g = torch.empty(2, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.energy(opt, ept, en_g, ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    comet.sync_status()
    # the block sums are atomic FP64 adds in arrival order: equal to rounding, not bitwise
    assert torch.allclose(en_g, en_eager, rtol=1e-13, atol=0)
