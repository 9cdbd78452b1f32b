"""Guard bands around every buffer the library touches (the sanitizer stand-in for the GPU pool,
where compute-sanitizer is closed): each input, output, workspace and pointer table lives in its
own device allocation between two 4 KiB bands of a canary byte, and after the call every band
must still hold the canary, every input must be unchanged bit for bit, and the result must
match the oracle.  Covers the split, FP64 and emulated-FP64 GEMM paths (exact and ragged tile
tails), a chain with a reduction and a batch label, the tensor-times-vector step, the three
transpose modes, the batched kernel in both result modes, the fused triples energy (tensor-core
and FMA paths), the host-buffer pipeline and the no-alloc entry point.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from helpers import normwise

pytestmark = pytest.mark.gpu

G = 4096          # guard bytes on each side
CANARY = 0xA5


@pytest.fixture(scope="module")
def comet():
    import paper_2102_06827_gb300 as c
    return c


class Guarded:
    """Device buffers between canary bands; check() verifies every band."""

    def __init__(self):
        self.parts = []

    def alloc(self, nbytes, dtype=None):
        import torch
        pad = (nbytes + 15) // 16 * 16
        full = torch.full((G + pad + G,), CANARY, dtype=torch.uint8, device="cuda")
        self.parts.append((full, nbytes))
        body = full[G:G + nbytes]
        return body if dtype is None else body.view(dtype)

    def put(self, arr, tdt):
        """a column-major numpy array copied into a guarded buffer of torch dtype tdt"""
        import torch
        flat = np.ravel(np.asarray(arr), order="F")
        t = self.alloc(flat.size * torch.empty(0, dtype=tdt).element_size(), tdt)
        t.copy_(torch.from_numpy(np.ascontiguousarray(flat)).to(tdt))
        return t

    def check(self):
        import torch
        torch.cuda.synchronize()
        for k, (full, n) in enumerate(self.parts):
            head = full[:G].cpu().numpy()
            tail = full[G + n:].cpu().numpy()
            assert (head == CANARY).all(), f"buffer {k}: band before it written"
            assert (tail == CANARY).all(), f"buffer {k}: band after it written ({int((tail != CANARY).sum())} bytes)"


def col(t, shape):
    a = t.cpu().numpy().astype(np.float64)
    return np.reshape(a, shape, order="F")


def labels_of(expr):
    _, out_labels, _, _, ops = oracle.parse(expr)
    return out_labels, [ls for _, ls in ops]


def run_contract(comet, expr, ext, precision, dtype, seed, **plan_kw):
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    out_labels, in_labels = labels_of(expr)
    arrays = [synth.tensor(tuple(ext[l] for l in ls), seed, t) for t, ls in enumerate(in_labels)]
    arrays = [a.astype(dtype).astype(np.float64) for a in arrays]
    g = Guarded()
    ins = [g.put(a, tdt) for a in arrays]
    before = [t.clone() for t in ins]
    out_shape = tuple(ext[l] for l in out_labels)
    n_out = int(np.prod(out_shape))
    out = g.alloc(n_out * torch.empty(0, dtype=tdt).element_size(), tdt)
    p = comet.Plan(expr, ext, tdt, precision=precision, **plan_kw)
    ws = g.alloc(p.workspace_bytes) if p.workspace_bytes else None
    p.contract(ins, out, ws)
    comet.sync_status()
    g.check()
    for a, b in zip(ins, before):
        assert torch.equal(a.view(torch.uint8), b.view(torch.uint8)), "an input was written"
    return col(out, out_shape), oracle.einsum(expr, *arrays), p


CCSD = "C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]"
TOL = {"split_bf16": 1e-6, "native": 1e-12, "emu_f64": 1e-12}


@pytest.mark.parametrize("precision,dtype", [("split_bf16", np.float32), ("native", np.float64),
                                             ("emu_f64", np.float64), ("native", np.float32)])
@pytest.mark.parametrize("ext", [dict(i=8, j=8, k=8, a=32, b=32, c=32),      # whole tiles
                                 dict(i=5, j=7, k=3, a=19, b=13, c=11)])    # ragged tails everywhere
def test_contract_bands(comet, precision, dtype, ext):
    got, ref, _ = run_contract(comet, CCSD, ext, precision, dtype, 61)
    tol = 2e-6 if (precision == "native" and dtype == np.float32) else TOL[precision]
    assert normwise(got, ref) <= tol


@pytest.mark.parametrize("precision,dtype", [("split_bf16", np.float32), ("native", np.float64)])
def test_chain_reduction_batch_bands(comet, precision, dtype):
    # x is summed inside A (a reduction step), b is on every operand and the result (batch)
    e = "D[i,l,b] = A[i,j,x,b] * B[j,k,b] * C[k,l,b]"
    ext = dict(i=21, j=17, x=5, b=3, k=19, l=23)
    got, ref, p = run_contract(comet, e, ext, precision, dtype, 62)
    assert len(p.info["steps"]) >= 3
    assert normwise(got, ref) <= TOL[precision]


@pytest.mark.parametrize("precision,dtype", [("split_bf16", np.float32), ("native", np.float64)])
def test_gemv_bands(comet, precision, dtype):
    e = "y[i,a] = A[c,d,i,a] * v[d,c]"
    ext = dict(c=37, d=29, i=11, a=13)
    got, ref, p = run_contract(comet, e, ext, precision, dtype, 63)
    assert any(s["kernel"] in ("gemv", "reduce") for s in p.info["steps"])
    assert normwise(got, ref) <= TOL[precision]


@pytest.mark.parametrize("extents,perm,dtype", [
    ((33, 27, 14), (2, 0, 1), np.float32),     # transposing tile kernel, odd runs
    ((40, 12, 18), (1, 2, 0), np.float64),     # transposing, 16-byte vectors
    ((17, 9, 5), (0, 2, 1), np.float32),       # copy mode, short odd run
    ((1001,), (0,), np.float32),               # a single run with a ragged tail
])
def test_transpose_bands(comet, extents, perm, dtype):
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    x = synth.tensor(extents, 64, 0).astype(dtype)
    g = Guarded()
    xi = g.put(x, tdt)
    before = xi.clone()
    out = g.alloc(x.size * x.itemsize, tdt)
    comet.transpose(xi, list(extents), list(perm), out=out)
    comet.sync_status()
    g.check()
    assert torch.equal(xi, before)
    ref = np.transpose(x, perm)
    got = np.reshape(out.cpu().numpy(), ref.shape, order="F")
    assert got.tobytes() == np.asfortranarray(ref).tobytes() or np.array_equal(got, ref)


@pytest.mark.parametrize("precision,dtype", [("split_bf16", np.float32), ("native", np.float64)])
def test_batched_bands(comet, precision, dtype):
    import torch
    from batched_data import EXPR, LABELS
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    ext = np.array([[5, 3, 7, 2, 4, 3, 9], [8, 8, 8, 8, 8, 8, 17], [1, 1, 1, 1, 1, 1, 1],
                    [11, 6, 9, 3, 5, 7, 33], [4, 9, 2, 6, 3, 8, 16]], dtype=np.int64)
    out_labels, in_labels = labels_of(EXPR)
    g = Guarded()
    host, ptrs, outs = [], [], []
    for b, row in enumerate(ext):
        e = dict(zip(LABELS, [int(x) for x in row]))
        pair = [synth.tensor(tuple(e[l] for l in ls), 65, 2 * b + t).astype(dtype).astype(np.float64)
                for t, ls in enumerate(in_labels)]
        host.append(pair)
        ptrs += [g.put(x, tdt).data_ptr() for x in pair]
        n = int(np.prod([e[l] for l in out_labels]))
        outs.append(g.alloc(n * torch.empty(0, dtype=tdt).element_size(), tdt))
    ptr_t = g.alloc(8 * len(ptrs), torch.int64)
    ptr_t.copy_(torch.tensor(ptrs, dtype=torch.int64))
    table = g.alloc(8 * len(outs), torch.int64)
    table.copy_(torch.tensor([t.data_ptr() for t in outs], dtype=torch.int64))
    plan = comet.BatchedPlan(EXPR, LABELS, ext, "f32" if dtype == np.float32 else "f64", precision=precision)
    ws = g.alloc(plan.workspace_bytes)
    plan.prepare(ws)
    res = g.alloc(16 * len(ext), torch.float64)
    plan.contract(ptr_t, res, ws, mode=0, key=1)
    plan.contract(ptr_t, table, ws, mode=1)
    comet.sync_status()
    g.check()
    tol = 1e-6 if dtype == np.float32 else 1e-12
    sums = res.cpu().numpy().reshape(-1, 2)
    for b in range(len(ext)):
        ref = oracle.einsum(EXPR, *host[b])
        T = col(outs[b], ref.shape)
        assert np.abs(T - ref).max() <= tol * max(np.abs(ref).max(), 1e-300), b
        q = float(np.sum(ref * ref))
        assert abs(sums[b, 1] - q) <= tol * q, b


@pytest.mark.parametrize("dtype,batch_rows", [(np.float32, None), (np.float32, "64"), (np.float64, None)])
def test_triples_energy_bands(comet, monkeypatch, dtype, batch_rows):
    # batch_rows "64": no block fits one batch of the tensor-core path, so the FMA kernel runs
    import torch
    from triples_terms import LABELS, SIGNS, block_inputs, terms
    if batch_rows:
        monkeypatch.setenv("COMET_TRIPLES_BATCH_ROWS", batch_rows)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    exts = [dict(a=9, b=5, c=6, i=7, j=3, k=5, d=11), dict(a=4, b=4, c=4, i=4, j=4, k=4, d=33),
            dict(a=1, b=2, c=1, i=3, j=1, k=2, d=1)]
    plan = comet.TriplesPlan(terms(), LABELS, [[e[l] for l in LABELS] for e in exts], SIGNS, tdt)
    g = Guarded()
    op_ptrs, eps_ptrs, refs = [], [], []
    for b, e in enumerate(exts):
        ops, eps = block_inputs(e, 66, b)
        ops = [tuple(x.astype(dtype).astype(np.float64) for x in pair) for pair in ops]
        eps = [x.astype(dtype).astype(np.float64) for x in eps]
        refs.append(oracle.triples_energy(terms(), ops, eps, SIGNS)[0])
        op_ptrs += [g.put(x, tdt).data_ptr() for pair in ops for x in pair]
        eps_ptrs += [g.put(x, tdt).data_ptr() for x in eps]
    opt = g.alloc(8 * len(op_ptrs), torch.int64)
    opt.copy_(torch.tensor(op_ptrs, dtype=torch.int64))
    ept = g.alloc(8 * len(eps_ptrs), torch.int64)
    ept.copy_(torch.tensor(eps_ptrs, dtype=torch.int64))
    en = g.alloc(8 * len(exts), torch.float64)
    ws = g.alloc(max(16, plan.workspace_bytes))
    plan.prepare(ws)
    plan.energy(opt, ept, en, ws)
    comet.sync_status()
    g.check()
    tol = 2e-5 if dtype == np.float32 else 1e-12
    got = en.cpu().numpy()
    for b in range(len(exts)):
        assert abs(got[b] - refs[b]) <= tol * abs(refs[b]), b


def test_host_pipeline_bands(comet):
    import torch
    ext = dict(i=16, j=14, k=16, a=46, b=44, c=48)
    out_labels, in_labels = labels_of(CCSD)
    arrays = [synth.tensor(tuple(ext[l] for l in ls), 67, t).astype(np.float32).astype(np.float64)
              for t, ls in enumerate(in_labels)]
    p = comet.Plan(CCSD, ext, torch.float32, precision="split_bf16", host_slices=3, host_slices_w=5)
    assert "host_pipe" in p.info
    g = Guarded()
    hin = [torch.from_numpy(np.ascontiguousarray(np.ravel(a, order="F")).astype(np.float32)).pin_memory()
           for a in arrays]
    din = [g.alloc(4 * t.numel(), torch.float32) for t in hin]
    out_shape = tuple(ext[l] for l in out_labels)
    n_out = int(np.prod(out_shape))
    hout = torch.empty(n_out, dtype=torch.float32).pin_memory()
    dout = g.alloc(4 * n_out, torch.float32)
    ws = g.alloc(p.workspace_bytes)
    p.contract_host_n([hin, hin], [hout, hout], din, dout, ws)
    g.check()
    assert normwise(col(hout, out_shape), oracle.einsum(CCSD, *arrays)) <= 1e-6


def test_noalloc_bands(comet):
    import torch
    ext = dict(i=5, j=7, k=3, a=19, b=13, c=11)
    out_labels, in_labels = labels_of(CCSD)
    arrays = [synth.tensor(tuple(ext[l] for l in ls), 68, t).astype(np.float32).astype(np.float64)
              for t, ls in enumerate(in_labels)]
    g = Guarded()
    ins = [g.put(a, torch.float32) for a in arrays]
    out_shape = tuple(ext[l] for l in out_labels)
    out = g.alloc(4 * int(np.prod(out_shape)), torch.float32)
    p = comet.Plan(CCSD, ext, torch.float32, precision="split_bf16")
    arr = (ctypes.c_void_p * len(ins))(*[t.data_ptr() for t in ins])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert comet.lib().comet_contract_noalloc(p._h, arr, ctypes.c_void_p(out.data_ptr()), stream) == 0
    comet.sync_status()
    g.check()
    assert normwise(col(out, out_shape), oracle.einsum(CCSD, *arrays)) <= 1e-6
