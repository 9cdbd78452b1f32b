"""GPU parity of the fused triples accumulation and energy (comet_triples_energy) against the
FP64 oracle (oracle.triples_energy: T as the sum of the nine permuted contraction terms,
E = sum T^2 / D).

Integer inputs make every product and partial sum of T exact in FP32 and FP64, so T is exact:
E then differs from the oracle's by the order of the FP64 sum (FP64 plans, relative 1e-12) or
by the FP32 rounding of each D, T^2 / D and of the 16-term FP32 partial sums (FP32 plans,
relative 1e-6).
Uniform inputs: FP64 within 1e-12, FP32 within 2e-5 relative per block (FP32 sums of 9 K
products per element; squared in E).
"""
import numpy as np
import pytest

import oracle
from triples_terms import LABELS, SIGNS, T_LABELS, block_inputs, terms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def comet():
    import paper_2102_06827_gb300 as c
    return c


def run(comet, exts, dtype, seed, kind="uniform", **kw):
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    ext_rows = [[e[l] for l in LABELS] for e in exts]
    plan = comet.TriplesPlan(terms(), LABELS, ext_rows, SIGNS, tdt)
    keep, op_ptrs, eps_ptrs, refs = [], [], [], []
    for b, e in enumerate(exts):
        ops, eps = block_inputs(e, seed, b, kind=kind, **kw)
        if dtype == np.float32:   # the oracle sees the values the GPU sees
            ops = [tuple(x.astype(np.float32).astype(np.float64) for x in pair) for pair in ops]
            eps = [x.astype(np.float32).astype(np.float64) for x in eps]
        refs.append(oracle.triples_energy(terms(), ops, eps, SIGNS)[0])
        for pair in ops:
            for x in pair:
                t = torch.from_numpy(np.ascontiguousarray(np.ravel(x, order="F"))).to(tdt).cuda()
                keep.append(t)
                op_ptrs.append(t.data_ptr())
        for x in eps:
            t = torch.from_numpy(np.asarray(x)).to(tdt).cuda()
            keep.append(t)
            eps_ptrs.append(t.data_ptr())
    opt = torch.tensor(op_ptrs, dtype=torch.int64, device="cuda")
    ept = torch.tensor(eps_ptrs, dtype=torch.int64, device="cuda")
    en = torch.empty(len(exts), dtype=torch.float64, device="cuda")
    ws = plan.workspace()
    plan.prepare(ws)
    plan.energy(opt, ept, en, ws)
    comet.sync_status()
    return en.cpu().numpy(), np.array(refs), plan


def rand_exts(n, seed, lo, hi, d_hi=None):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        e = {l: int(rng.integers(lo, hi + 1)) for l in T_LABELS}
        e["d"] = int(rng.integers(lo, (d_hi or hi) + 1))
        out.append(e)
    return out


SHAPES = [
    [dict(a=4, b=4, c=4, i=4, j=4, k=4, d=4)],                        # one tile
    [dict(a=5, b=6, c=7, i=3, j=2, k=9, d=5), dict(a=1, b=1, c=1, i=1, j=1, k=1, d=1)],
    [dict(a=8, b=5, c=6, i=4, j=7, k=3, d=40)],                       # the summed label in two passes
]


@pytest.mark.parametrize("exts", SHAPES + [rand_exts(6, 7, 1, 9)])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_integers_exact(comet, exts, dtype):
    got, ref, _ = run(comet, exts, dtype, 3, kind="int", lo=-3, hi=3)
    tol = 1e-12 if dtype == np.float64 else 1e-6
    assert np.all(np.abs(got - ref) <= tol * np.abs(ref) + 1e-300)


@pytest.mark.parametrize("exts", SHAPES + [rand_exts(8, 8, 2, 11, d_hi=36)])
@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 2e-5)])
def test_uniform(comet, exts, dtype, tol):
    got, ref, plan = run(comet, exts, dtype, 4)
    assert plan.info["triples"] and plan.info["terms"] == 9
    assert np.all(ref < 0)
    assert np.all(np.abs(got - ref) <= tol * np.abs(ref))


def test_fp32_withheld_load_times_out_and_context_survives(comet, monkeypatch):
    # fault injection on the host side of the tensor-core path: one ring slot's operand loads
    # are withheld, the MMA thread's bounded wait runs out, the status word reports it, and the
    # next launch on the same context is correct
    exts = SHAPES[1]
    monkeypatch.setenv("COMET_TRIPLES_DEBUG", "1")
    monkeypatch.setenv("COMET_WAIT_TIMEOUT_MS", "100")
    with pytest.raises(comet.CometError) as err:
        run(comet, exts, np.float32, 3)
    assert err.value.name == "COMET_ERR_TIMEOUT"
    monkeypatch.delenv("COMET_TRIPLES_DEBUG")
    monkeypatch.delenv("COMET_WAIT_TIMEOUT_MS")
    got, ref, plan = run(comet, exts, np.float32, 3)
    assert plan.info["tensor_core"]
    assert np.all(np.abs(got - ref) <= 2e-5 * np.abs(ref))


@pytest.mark.parametrize("route", ["batches", "fma"])
def test_fp32_routes(comet, monkeypatch, route):
    # the FP32 tensor-core path with one batch per block, and the FP32 FMA kernel (a batch cap
    # below every block), against the oracle: integers and uniform inputs
    exts = SHAPES[1] + SHAPES[2] + rand_exts(3, 17, 2, 12, d_hi=40)
    monkeypatch.setenv("COMET_TRIPLES_BATCH_ROWS", "40000" if route == "batches" else "1000")
    got, ref, plan = run(comet, exts, np.float32, 3, kind="int", lo=-3, hi=3)
    assert plan.info["tensor_core"] == (route == "batches")
    if route == "batches":
        assert plan.info["batches"] > 1
    assert np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref) + 1e-300)
    got, ref, _ = run(comet, exts, np.float32, 4)
    assert np.all(np.abs(got - ref) <= 2e-5 * np.abs(ref))


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 1e-5)])
def test_terms_add_linearly(comet, dtype, tol):
    # the same block with terms 0..3 each split into two halves (13 terms) gives the same energy
    # (alpha = 0.5 scales the X entries in shared memory)
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    e = dict(a=6, b=5, c=7, i=4, j=6, k=5, d=9)
    ops, eps = block_inputs(e, 5, 0)
    t9 = terms()
    half = [s.replace("= ", "= 0.5 * ", 1) for s in t9[:4]]
    split_terms = half + half + t9[4:]
    split_ops = ops[:4] + ops[:4] + ops[4:]
    res = []
    for tl, ol in ((t9, ops), (split_terms, split_ops)):
        plan = comet.TriplesPlan(tl, LABELS, [[e[l] for l in LABELS]], SIGNS, tdt)
        keep, ptrs = [], []
        for pair in ol:
            for x in pair:
                t = torch.from_numpy(np.ascontiguousarray(np.ravel(x, order="F"))).to(tdt).cuda()
                keep.append(t)
                ptrs.append(t.data_ptr())
        ept = [torch.from_numpy(np.asarray(x)).to(tdt).cuda() for x in eps]
        en = torch.empty(1, dtype=torch.float64, device="cuda")
        ws = plan.workspace()
        plan.prepare(ws)
        plan.energy(torch.tensor(ptrs, dtype=torch.int64, device="cuda"),
                    torch.tensor([t.data_ptr() for t in ept], dtype=torch.int64, device="cuda"), en, ws)
        comet.sync_status()
        res.append(float(en.item()))
    assert abs(res[0] - res[1]) <= tol * abs(res[0])


def test_full_workload_sampled(comet):
    # the 4096-block workload the bench times (extents uniform 8..32, seed 3; operands uniform
    # [-1, 1) from seed 11 in one device buffer; eps in [1, 2) and [-2, -1)), FP32 on the tensor
    # cores in one call: every energy finite and negative (D < 0 everywhere), and the two smallest
    # blocks and the median-sized one within 2e-5 of the oracle on the values the GPU read
    import torch
    import synth
    tl = terms()
    col = {l: q for q, l in enumerate(LABELS)}
    ext = synth.triples_blocks(4096)
    opl = [[tuple(col[l] for l in ls) for ls in pair] for pair in
           [[oracle.parse(e)[4][0][1], oracle.parse(e)[4][1][1]] for e in tl]]
    sizes = np.array([int(np.prod(ext[b, list(c)])) for b in range(len(ext)) for pair in opl for c in pair],
                     dtype=np.int64)
    buf = torch.empty(int(sizes.sum()), dtype=torch.float32, device="cuda")
    chunk = 1 << 27
    for c0 in range(0, buf.numel(), chunk):
        n = min(chunk, buf.numel() - c0)
        buf[c0:c0 + n] = synth.torch_uniform(11, c0 // chunk, n, "cuda").float()
    starts = np.concatenate([[0], np.cumsum(sizes)])
    ops = torch.tensor(starts[:-1] * 4, dtype=torch.int64, device="cuda") + buf.data_ptr()
    e_sizes = np.array([int(ext[b, col[l]]) for b in range(len(ext)) for l in T_LABELS], dtype=np.int64)
    e_starts = np.concatenate([[0], np.cumsum(e_sizes)])
    shift = np.concatenate([np.full(n, 1.5 if q % 6 < 3 else -1.5) for q, n in enumerate(e_sizes)])
    ebuf = (synth.torch_uniform(12, 0, int(e_sizes.sum()), "cuda") * 0.5 + torch.from_numpy(shift).cuda()).float()
    eps = torch.tensor(e_starts[:-1] * 4, dtype=torch.int64, device="cuda") + ebuf.data_ptr()
    plan = comet.TriplesPlan(tl, LABELS, ext, SIGNS, torch.float32)
    assert plan.info["tensor_core"]
    ws = plan.workspace()
    plan.prepare(ws)
    en = torch.empty(len(ext), dtype=torch.float64, device="cuda")
    plan.energy(ops, eps, en, ws)
    comet.sync_status()
    got = en.cpu().numpy()
    assert np.all(np.isfinite(got)) and np.all(got < 0)
    t_size = np.prod(ext[:, :6], axis=1)
    order = np.argsort(t_size, kind="stable")
    per_block = 2 * len(tl)
    for b in [int(order[0]), int(order[1]), int(order[len(order) // 2])]:
        host_ops = []
        for p, pair in enumerate(opl):
            xs = []
            for q, c in enumerate(pair):
                k = b * per_block + 2 * p + q
                v = buf[int(starts[k]):int(starts[k + 1])].double().cpu().numpy()
                xs.append(np.reshape(v, [int(ext[b, i]) for i in c], order="F"))
            host_ops.append(tuple(xs))
        host_eps = [ebuf[int(e_starts[b * 6 + q]):int(e_starts[b * 6 + q + 1])].double().cpu().numpy()
                    for q in range(6)]
        ref = oracle.triples_energy(tl, host_ops, host_eps, SIGNS)[0]
        assert abs(got[b] - ref) <= 2e-5 * abs(ref), (b, got[b], ref)
    del buf, ebuf, ws
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 2e-5)])
def test_medium_blocks_of_the_workload_range(comet, dtype, tol):
    # blocks from the middle of the workload's extent range (16..20 per label): the FP64 FMA
    # kernel's 4 x 4 register tiles and the FP32 tensor-core path's pair-tiles with ragged
    # edges along every label, against the oracle
    exts = [dict(a=17, b=19, c=16, i=18, j=20, k=17, d=19), dict(a=20, b=16, c=18, i=17, j=16, k=19, d=33)]
    got, ref, plan = run(comet, exts, dtype, 5)
    assert np.all(np.abs(got - ref) <= tol * np.abs(ref))
