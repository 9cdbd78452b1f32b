"""GPU parity of comet_contract_host (host buffers in, host buffer out) against the FP64 oracle.

Covers the slice pipeline of one-step split and emulated-FP64 plans (pinned host buffers: the
larger operand crosses in slices along the last label of its GEMM row group, overlapped with the
GEMMs of the previous slices) and the serial path (pageable buffers, or host_slices=1).  Bars as
for comet_contract: split path within 1e-6 normwise, emulated FP64 within 1e-12, integer
inputs bit-exact on the split path.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import normwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def comet():
    import paper_2102_06827_gb300 as c
    return c


def host_col(a, dtype, pinned):
    """numpy array -> CPU torch tensor holding it column-major (pinned or pageable)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(np.asfortranarray(np.asarray(a, dtype=dtype)).T))
    return t.pin_memory() if pinned else t.clone()


def run_host(comet, expr, ext, arrays, dtype, precision, pinned=True, out_init=None, **kw):
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    p = comet.Plan(expr, ext, tdt, precision=precision, **kw)
    _, out_labels, _, _, _ = oracle.parse(expr)
    out_shape = tuple(ext[l] for l in out_labels)
    init = np.zeros(out_shape) if out_init is None else out_init
    hin = [host_col(a, dtype, pinned) for a in arrays]
    hout = host_col(init, dtype, pinned)
    din = [torch.full(t.shape, float("nan"), dtype=tdt, device="cuda") for t in hin]
    dout = torch.full(hout.shape, float("nan"), dtype=tdt, device="cuda")
    p.contract_host(hin, hout, din, dout, p.workspace())
    return np.asfortranarray(hout.numpy().T), p, dout


def inputs(expr, ext, seed, kind="uniform", **kw):
    _, _, _, _, ops = oracle.parse(expr)
    return [synth.tensor(tuple(ext[l] for l in ls), seed, t, kind=kind, **kw) for t, (_, ls) in enumerate(ops)]


CCSD = "C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]"


@pytest.mark.parametrize("slices,w_slices,ext", [
    (4, 1, dict(i=16, j=16, k=16, a=48, b=48, c=48)),     # equal slices
    (4, 1, dict(i=16, j=18, k=16, a=48, b=40, c=48)),     # A larger: slices of a (M group)
    (4, 1, dict(i=16, j=18, k=16, a=40, b=48, c=48)),     # chunk 5, short last slice of 3
    (16, 1, dict(i=8, j=16, k=8, a=40, b=24, c=40)),      # one unit of the label per slice
    (4, 4, dict(i=16, j=16, k=16, a=48, b=48, c=48)),     # both operands in slices
    (3, 5, dict(i=16, j=14, k=16, a=46, b=44, c=48)),     # both ragged
])
def test_pipeline_split(comet, slices, w_slices, ext):
    A, B = inputs(CCSD, ext, 3)
    C, p, dout = run_host(comet, CCSD, ext, [A, B], np.float32, "split_bf16", host_slices=slices,
                          host_slices_w=w_slices)
    hp = p.info.get("host_pipe")
    step = p.info["steps"][0]
    assert hp is not None and hp["slices"] * hp["w_slices"] > 1
    assert hp["w_slices"] == min(w_slices, ext[hp["w_label"]]) or w_slices == 1
    assert hp["label"] == (step["N"] if hp["side"] == "N" else step["M"])[-1]
    assert hp["w_label"] == (step["M"] if hp["side"] == "N" else step["N"])[-1]
    assert normwise(C, oracle.einsum(CCSD, A, B)) <= 1e-6
    # the device output holds the result as well
    import torch
    assert torch.equal(dout.cpu(), host_col(C, np.float32, False))


@pytest.mark.parametrize("expr,blockwise", [
    ("C[j,i,c] = A[i,k,c] * B[k,j]", False),   # a label between the two sliced ones: column copies
    ("C[c,i,j] = A[i,k,c] * B[k,j]", True),    # the W label next to the sliced one: block copies
])
def test_pipeline_copy_out_routes(comet, expr, blockwise):
    ext = dict(i=40, c=24, k=32, j=20)
    A, B = inputs(expr, ext, 11)
    C, p, _ = run_host(comet, expr, ext, [A, B], np.float32, "split_bf16", host_slices=3, host_slices_w=2)
    hp = p.info["host_pipe"]
    assert hp["blockwise"] == blockwise and hp["slices"] == 3 and hp["w_slices"] == 2
    assert normwise(C, oracle.einsum(expr, A, B)) <= 1e-6


def test_pipeline_integers_exact_and_equal_to_device_path(comet):
    ext = dict(i=16, j=12, k=16, a=32, b=48, c=32)
    A, B = inputs(CCSD, ext, 4, kind="int", lo=-3, hi=3)
    C, p, _ = run_host(comet, CCSD, ext, [A, B], np.float32, "split_bf16", host_slices=3)
    assert p.info["host_pipe"]["slices"] == 3
    ref = oracle.einsum(CCSD, A, B)
    assert np.array_equal(C, ref)


def test_pipeline_sliced_m_operand(comet):
    # A is the larger operand: the slices run along m, the last label of the M group
    e = "C[m,n] = A[m,k] * B[k,n]"
    ext = dict(m=600, n=136, k=72)
    A, B = inputs(e, ext, 5)
    C, p, _ = run_host(comet, e, ext, [A, B], np.float32, "split_bf16", host_slices=3, host_slices_w=2)
    hp = p.info["host_pipe"]
    assert hp["side"] == "M" and hp["label"] == "m" and hp["slices"] == 3
    assert hp["w_label"] == "n" and hp["w_slices"] == 2
    assert normwise(C, oracle.einsum(e, A, B)) <= 1e-6


def test_pipeline_accumulate_alpha(comet):
    e = "C[i,j] += 0.5 * A[i,k] * B[k,j]"
    ext = dict(i=300, j=520, k=96)
    A, B = inputs(e, ext, 6)
    C0 = synth.tensor((300, 520), 6, 9).astype(np.float32).astype(np.float64)
    C, p, _ = run_host(comet, e, ext, [A, B], np.float32, "split_bf16", out_init=C0, host_slices=4,
                       host_slices_w=3)
    assert p.info["host_pipe"]["slices"] == 4 and p.info["host_pipe"]["w_slices"] == 3
    ref = oracle.einsum(e, A, B, out=np.asfortranarray(C0.copy()))
    assert normwise(C, ref) <= 2e-6


def test_pipeline_emulated_f64(comet):
    ext = dict(i=8, j=20, k=8, a=40, b=24, c=40)
    A, B = inputs(CCSD, ext, 7)
    C, p, _ = run_host(comet, CCSD, ext, [A, B], np.float64, "emu_f64", host_slices=3, host_slices_w=2)
    assert p.info["host_pipe"]["slices"] == 3 and p.info["host_pipe"]["w_slices"] == 2
    assert normwise(C, oracle.einsum(CCSD, A, B)) <= 1e-12


@pytest.mark.parametrize("pinned,slices", [(False, 4), (True, 1)])
def test_serial_path(comet, pinned, slices):
    # pageable host buffers, or slicing switched off: copies, contraction and copy back in order
    ext = dict(i=16, j=16, k=16, a=48, b=48, c=48)
    A, B = inputs(CCSD, ext, 8)
    C, p, _ = run_host(comet, CCSD, ext, [A, B], np.float32, "split_bf16", pinned=pinned,
                       host_slices=slices)
    assert ("host_pipe" in p.info) == (slices != 1)
    assert normwise(C, oracle.einsum(CCSD, A, B)) <= 1e-6


def test_serial_multi_step_and_native(comet):
    e = "D[i,l] = A[i,j] * B[j,k] * C[k,l]"
    ext = dict(i=40, j=50, k=60, l=30)
    arrays = inputs(e, ext, 9)
    D, p, _ = run_host(comet, e, ext, arrays, np.float64, "native")
    assert "host_pipe" not in p.info
    assert normwise(D, oracle.einsum(e, *arrays)) <= 1e-12


def run_host_n(comet, expr, ext, sets, dtype, precision, pinned=True, out_inits=None, shared_out=False, **kw):
    """comet_contract_host_n over len(sets) input sets; returns the host results (one per call, or
    the one shared buffer), the plan and the per-call results of single comet_contract_host calls
    on the same plan."""
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    p = comet.Plan(expr, ext, tdt, precision=precision, **kw)
    _, out_labels, _, _, _ = oracle.parse(expr)
    out_shape = tuple(ext[l] for l in out_labels)
    inits = out_inits or [np.zeros(out_shape)] * len(sets)
    hin = [[host_col(a, dtype, pinned) for a in arrays] for arrays in sets]
    houts = [host_col(inits[0], dtype, pinned)] * len(sets) if shared_out else \
        [host_col(c, dtype, pinned) for c in inits]
    din = [torch.full(t.shape, float("nan"), dtype=tdt, device="cuda") for t in hin[0]]
    dout = torch.full(houts[0].shape, float("nan"), dtype=tdt, device="cuda")
    p.contract_host_n(hin, houts, din, dout, p.workspace())
    got = [np.asfortranarray(h.numpy().T).copy() for h in houts]
    single = []
    for t, arrays in enumerate(hin):   # the same plan, one call per input set
        h1 = host_col(inits[t], dtype, pinned)
        p.contract_host(arrays, h1, din, dout, p.workspace())
        single.append(np.asfortranarray(h1.numpy().T).copy())
    return got, p, single


@pytest.mark.parametrize("expr,ext,slices,w_slices", [
    (CCSD, dict(i=16, j=16, k=16, a=48, b=48, c=48), 4, 4),          # block copies back
    ("C[j,i,c] = A[i,k,c] * B[k,j]", dict(i=40, c=24, k=32, j=20), 3, 2),   # column copies back
    (CCSD, dict(i=16, j=14, k=16, a=46, b=44, c=48), 3, 5),          # both ragged
])
def test_pipelined_calls(comet, expr, ext, slices, w_slices):
    # three calls with their own inputs and outputs: each equals its single call bit for bit
    sets = [inputs(expr, ext, 20 + t) for t in range(3)]
    got, p, single = run_host_n(comet, expr, ext, sets, np.float32, "split_bf16", host_slices=slices,
                                host_slices_w=w_slices)
    assert p.info["host_pipe"]["slices"] == slices
    for t, arrays in enumerate(sets):
        assert np.array_equal(got[t], single[t])
        assert normwise(got[t], oracle.einsum(expr, *arrays)) <= 1e-6


def test_pipelined_calls_shared_output_and_integers(comet):
    # integer inputs (exact on the split path); one host output for all calls ends with the last
    ext = dict(i=16, j=12, k=16, a=32, b=48, c=32)
    sets = [inputs(CCSD, ext, 30 + t, kind="int", lo=-3, hi=3) for t in range(4)]
    got, p, single = run_host_n(comet, CCSD, ext, sets, np.float32, "split_bf16", shared_out=True,
                                host_slices=3, host_slices_w=2)
    assert np.array_equal(got[-1], oracle.einsum(CCSD, *sets[-1]))
    assert np.array_equal(single[0], oracle.einsum(CCSD, *sets[0]))


def test_pipelined_calls_accumulate(comet):
    e = "C[i,j] += 0.5 * A[i,k] * B[k,j]"
    ext = dict(i=300, j=520, k=96)
    sets = [inputs(e, ext, 40 + t) for t in range(3)]
    inits = [synth.tensor((300, 520), 41, t).astype(np.float32).astype(np.float64) for t in range(3)]
    got, p, single = run_host_n(comet, e, ext, sets, np.float32, "split_bf16", out_inits=inits, host_slices=4,
                                host_slices_w=3)
    for t, arrays in enumerate(sets):
        assert np.array_equal(got[t], single[t])
        ref = oracle.einsum(e, *arrays, out=np.asfortranarray(inits[t].copy()))
        assert normwise(got[t], ref) <= 2e-6


def test_pipelined_calls_emulated_and_serial(comet):
    ext = dict(i=8, j=20, k=8, a=40, b=24, c=40)
    sets = [inputs(CCSD, ext, 50 + t) for t in range(2)]
    got, p, _ = run_host_n(comet, CCSD, ext, sets, np.float64, "emu_f64", host_slices=3, host_slices_w=2)
    assert "host_pipe" in p.info
    for t, arrays in enumerate(sets):
        assert normwise(got[t], oracle.einsum(CCSD, *arrays)) <= 1e-12
    # pageable buffers: the calls run one after another on the stream
    got, p, single = run_host_n(comet, CCSD, ext, sets, np.float32, "split_bf16", pinned=False, host_slices=3)
    for t, arrays in enumerate(sets):
        assert np.array_equal(got[t], single[t])
        assert normwise(got[t], oracle.einsum(CCSD, *arrays)) <= 1e-6


def test_calls_of_a_chain_run_in_order(comet):
    # a multi-step plan has no slice pipeline: the calls run one after another on the stream,
    # each equal to its single call and to the oracle
    e = "D[i,l] = A[i,j] * B[j,k] * C[k,l]"
    ext = dict(i=40, j=50, k=60, l=30)
    sets = [inputs(e, ext, 60 + t) for t in range(3)]
    got, p, single = run_host_n(comet, e, ext, sets, np.float64, "native")
    assert "host_pipe" not in p.info
    for t, arrays in enumerate(sets):
        assert np.array_equal(got[t], single[t])
        assert normwise(got[t], oracle.einsum(e, *arrays)) <= 1e-12
