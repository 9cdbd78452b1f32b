"""GPU parity of views (slices lo:step of stored tensors, comet_plan_views) and diagonals (a
label written twice inside one tensor) against the FP64 oracle on the same slices.

The oracle sees the slice as numpy cuts it out of the stored array, so the library's stride and
offset arithmetic is checked against numpy's.  Outside an output view the stored tensor must be
untouched (bit-exact).  Bars as elsewhere: FP64 1e-12, split 1e-6, emulated FP64 1e-12 normwise.
"""
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


def cut(a, spec):
    """numpy slice of a stored array: spec = [(dim, lo, step, n), ...]"""
    idx = [slice(None)] * a.ndim
    for d, lo, st, n in spec:
        idx[d] = slice(lo, lo + (n - 1) * st + 1, st)
    return a[tuple(idx)]


def run_views(comet, expr, ext, stores, out_store, views, dtype, precision="native"):
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    p = comet.Plan(expr, ext, tdt, precision=precision, views=views)
    ins = [to_dev(a, dtype) for a in stores]
    out = to_dev(out_store, dtype)
    p.contract(ins, out, p.workspace())
    comet.sync_status()
    return from_dev(out), p


def specs_of(views, n_t, ext_of_dim):
    """views -> per tensor numpy cut specs [(dim, lo, step, n)]"""
    s = [[] for _ in range(n_t)]
    for o, d, _, lo, st in views:
        s[o].append((d, lo, st, ext_of_dim(o, d)))
    return s


CASES = [
    # expression, extents, views (operand, dim, declared, lo, step), stored shapes
    ("C[i,j] = A[i,k] * B[k,j]", dict(i=70, j=90, k=50),
     [(0, 0, 160, 3, 2), (1, 0, 64, 7, 1), (2, 1, 200, 5, 2)],
     [(160, 50), (64, 90), (70, 200)]),
    ("C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]", dict(i=6, j=5, k=7, a=20, b=18, c=9),
     [(0, 1, 41, 1, 2), (1, 3, 11, 2, 1), (2, 0, 8, 1, 1), (2, 3, 40, 3, 2)],
     [(7, 41, 9, 6), (9, 18, 7, 11), (8, 20, 5, 40)]),
    ("y[r] = M[c,r] * x[c]", dict(r=300, c=257),
     [(0, 1, 601, 1, 2), (1, 0, 900, 11, 3)],
     [(257, 601), (900,), (300,)]),
    ("C[i,j,b] = A[i,k,b] * B[k,j,b]", dict(i=33, j=17, k=40, b=5),
     [(0, 2, 9, 0, 2), (1, 0, 45, 5, 1)],
     [(33, 40, 9), (45, 17, 5), (33, 17, 5)]),
]


@pytest.mark.parametrize("expr,ext,views,shapes", CASES)
@pytest.mark.parametrize("dtype,precision,tol", [(np.float64, "native", 1e-12),
                                                 (np.float32, "split_bf16", 1e-6),
                                                 (np.float64, "emu_f64", 1e-12)])
def test_views_match_oracle_on_numpy_slices(comet, expr, ext, views, shapes, dtype, precision, tol):
    _, out_labels, _, _, ops = oracle.parse(expr)
    labels = [ls for _, ls in ops] + [out_labels]
    n_t = len(labels)
    stores = [synth.tensor(shp, 21, t) for t, shp in enumerate(shapes[:-1])]
    out_store = synth.tensor(shapes[-1], 21, 9)
    if dtype == np.float32:
        stores = [s.astype(np.float32).astype(np.float64) for s in stores]
        out_store = out_store.astype(np.float32).astype(np.float64)
    # outside the views the stored inputs hold values far larger than inside: an operand scale
    # taken over the stored tensor instead of the view would fail the split bar
    spec = specs_of(views, n_t, lambda o, d: ext[labels[o][d]])
    for t in range(n_t - 1):
        big = np.full(shapes[t], 3.0e4)
        view = cut(stores[t], spec[t]).copy()
        stores[t] = np.asfortranarray(big)
        cut(stores[t], spec[t])[...] = view
    C, p = run_views(comet, expr, ext, stores, out_store, views, dtype, precision)
    assert "views" in p.info
    ins = [cut(stores[t], spec[t]) for t in range(n_t - 1)]
    ref = oracle.einsum(expr, *[np.asfortranarray(a) for a in ins])
    got = cut(C, spec[-1])
    assert normwise(got, ref) <= tol
    # outside the output view nothing changed
    mask = np.ones(shapes[-1], dtype=bool)
    cut(mask, spec[-1])[...] = False
    assert np.array_equal(C[mask], np.asarray(out_store, dtype=dtype)[mask])


def test_view_copy_and_transpose_bit_exact_with_odd_offsets(comet):
    # offsets of one element: the copy kernels must fall back from 16-byte accesses
    e = "B[j,i] = A[i,j]"
    ext = dict(i=129, j=67)
    views = [(0, 0, 131, 1, 1), (0, 1, 70, 3, 1), (1, 0, 69, 1, 1)]
    A = synth.tensor((131, 70), 22, 0).astype(np.float32)
    B0 = synth.tensor((69, 129), 22, 1).astype(np.float32)
    B, p = run_views(comet, e, ext, [A], B0, views, np.float32)
    assert p.info["steps"][0]["kernel"] == "copy"
    ref = cut(A, [(0, 1, 1, 129), (1, 3, 1, 67)]).T
    assert np.array_equal(B[1:68, :], ref)
    assert np.array_equal(B[[0, 68], :], B0[[0, 68], :])
    # identity copy of a strided slice into a strided slice (copy mode, element-wise)
    e = "D[i,j] = A[i,j]"
    views = [(0, 0, 131, 2, 1), (0, 1, 70, 0, 1), (1, 0, 130, 1, 1), (1, 1, 68, 1, 1)]
    D0 = synth.tensor((130, 68), 22, 2).astype(np.float32)
    D, _ = run_views(comet, e, ext, [A], D0, views, np.float32)
    assert np.array_equal(D[1:, 1:], A[2:, :67])
    assert np.array_equal(D[0, :], D0[0, :]) and np.array_equal(D[:, 0], D0[:, 0])


DIAG = [
    ("t[] = A[i,i]", dict(i=37), [(37, 37)]),
    ("c[i] = A[i,i]", dict(i=300), [(300, 300)]),
    ("v[i] = A[i,i] * x[i]", dict(i=257), [(257, 257), (257,)]),
    ("C[i,j] = A[i,k,k] * B[k,j]", dict(i=40, j=30, k=24), [(40, 24, 24), (24, 30)]),
    ("D[i,i] = A[i,k] * B[k,i]", dict(i=48, k=64), [(48, 64), (64, 48)]),
]


@pytest.mark.parametrize("expr,ext,shapes", DIAG)
@pytest.mark.parametrize("dtype,precision", [(np.float64, "native"), (np.float32, "split_bf16")])
def test_diagonals_integers_exact(comet, expr, ext, shapes, dtype, precision):
    import torch
    arrays = [synth.tensor(s, 23, t, kind="int", lo=-3, hi=3) for t, s in enumerate(shapes)]
    _, out_labels, _, _, _ = oracle.parse(expr)
    out_shape = tuple(ext[l] for l in out_labels)
    out0 = np.full(out_shape, 7.0)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    p = comet.Plan(expr, ext, tdt, precision=precision)
    ins = [to_dev(a, dtype) for a in arrays]
    out = to_dev(out0, dtype) if out_shape else torch.full((), 7.0, dtype=tdt, device="cuda")
    p.contract(ins, out, p.workspace())
    comet.sync_status()
    C = from_dev(out)
    # the oracle takes repeated labels by definition (pinned against np.trace); an output
    # diagonal is written element by element, the rest of the stored output kept
    if expr.startswith("D[i,i]"):
        ref = np.full(out_shape, 7.0)
        d = oracle.einsum("d[i] = A[i,k] * B[k,i]", *arrays)
        ref[np.arange(48), np.arange(48)] = d
    else:
        ref = oracle.einsum(expr, *arrays)
    assert np.array_equal(np.asarray(C, dtype=np.float64), np.asarray(ref, dtype=np.float64))


def test_views_through_the_host_entry_point(comet):
    # the host entry point copies the stored tensors whole (serial path: no slice pipeline on
    # views) and writes back the stored output with the elements outside the view unchanged
    import torch
    e = "C[i,j] = A[i,k] * B[k,j]"
    ext = dict(i=70, j=90, k=50)
    views = [(0, 0, 160, 3, 2), (2, 1, 200, 5, 2)]
    A = synth.tensor((160, 50), 24, 0).astype(np.float32)
    B = synth.tensor((50, 90), 24, 1).astype(np.float32)
    C0 = synth.tensor((70, 200), 24, 2).astype(np.float32)
    p = comet.Plan(e, ext, torch.float32, precision="split_bf16", views=views)
    assert "host_pipe" not in p.info
    ref = oracle.einsum(e, np.asfortranarray(A.astype(np.float64)[3:3 + 69 * 2 + 1:2, :]), B.astype(np.float64))

    def host(a):
        return torch.from_numpy(np.ascontiguousarray(np.asfortranarray(a).T)).pin_memory()
    hA, hB, hC = host(A), host(B), host(C0)
    p.contract_host([hA, hB], hC, [torch.empty_like(hA, device="cuda"), torch.empty_like(hB, device="cuda")],
                    torch.empty_like(hC, device="cuda"), p.workspace())
    C = np.asfortranarray(hC.numpy().T)
    assert normwise(C[:, 5:5 + 89 * 2 + 1:2], ref) <= 1e-6
    mask = np.ones((70, 200), dtype=bool)
    mask[:, 5:5 + 89 * 2 + 1:2] = False
    assert np.array_equal(C[mask], C0[mask])
