"""GPU parity of comet_transpose against the oracle's bit-move transpose (bit-exact)."""
import itertools

import numpy as np
import pytest

import oracle
import synth
from helpers import from_dev, same_bits, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def comet():
    import paper_2102_06827_gb300 as c
    return c


def run(comet, a, perm):
    x = to_dev(a)
    out = comet.transpose(x, a.shape, perm)
    comet.sync_status()
    return from_dev(out)


def test_extent24_fp64_perm_201(comet):
    # the extent-24 FP64 workload: A[a,e,b] of 24^3 by (2,0,1), bit-exact
    A = synth.tensor((24, 24, 24), 0, 0)
    T = run(comet, A, (2, 0, 1))
    assert T.tobytes(order="F") == oracle.transpose(A, (2, 0, 1)).tobytes(order="F")


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("perm", list(itertools.permutations(range(4))))
def test_rank4_all_perms_ragged(comet, dtype, perm):
    A = synth.tensor((7, 8, 5, 12), 1, 0, dtype=dtype)
    T = run(comet, A, perm)
    assert T.tobytes(order="F") == oracle.transpose(A, perm).tobytes(order="F")


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("case", range(8))
def test_rank6_random_perms(comet, dtype, case):
    rng = np.random.default_rng(100 + case)
    perm = tuple(int(p) for p in rng.permutation(6))
    ext = tuple(int(e) for e in synth.uniform_extents(7, case, 6, 2, 9))
    A = synth.tensor(ext, 2, case, dtype=dtype)
    T = run(comet, A, perm)
    assert T.tobytes(order="F") == oracle.transpose(A, perm).tobytes(order="F")


def test_special_bit_patterns_survive(comet):
    bits = synth.raw_bits(3, 0, 0, 6 * 10 * 9)
    A = np.asfortranarray(bits.view(np.float64).reshape((6, 10, 9), order="F")).copy(order="F")
    flat = A.reshape(-1, order="F")
    flat[:5] = [np.nan, -0.0, 5e-324, -np.inf, 1e-310]
    A = np.asfortranarray(flat.reshape((6, 10, 9), order="F"))
    T = run(comet, A, (1, 2, 0))
    assert T.tobytes(order="F") == oracle.transpose(A, (1, 2, 0)).tobytes(order="F")
    A32 = np.asfortranarray(bits.astype(np.uint32).view(np.float32).reshape((6, 10, 9), order="F"))
    T32 = run(comet, A32, (2, 0, 1))
    assert T32.tobytes(order="F") == oracle.transpose(A32, (2, 0, 1)).tobytes(order="F")


@pytest.mark.parametrize("shape,perm", [((1,), (0,)), ((5, 1, 3), (1, 2, 0)), ((1, 1, 1), (2, 1, 0)),
                                         ((300, 7), (1, 0)), ((8, 8, 8, 8, 8, 8), (5, 4, 3, 2, 1, 0)),
                                         ((64, 3, 64), (2, 1, 0)), ((9, 130, 70), (0, 2, 1))])
def test_edge_shapes(comet, shape, perm):
    for dtype in (np.float32, np.float64):
        A = synth.tensor(shape, 4, 0, dtype=dtype)
        T = run(comet, A, perm)
        assert T.tobytes(order="F") == oracle.transpose(A, perm).tobytes(order="F")


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_64mib_rank4(comet, dtype):
    # a size of the transpose sweep: 64 MiB, many tiles, full comparison
    n = (64 << 20) // np.dtype(dtype).itemsize
    ext = (32, 64, 64, n // (32 * 64 * 64))
    A = synth.tensor(ext, 5, 0, dtype=dtype)
    for perm in [(1, 3, 0, 2), (3, 2, 1, 0), (0, 2, 1, 3)]:
        T = run(comet, A, perm)
        assert same_bits(T, oracle.transpose(A, perm))


def test_rejects_bad_arguments(comet):
    import torch
    x = torch.zeros(16, device="cuda")
    with pytest.raises(comet.CometError) as e:
        comet.transpose(x, [4, 4], [1, 1])
    assert e.value.name == "COMET_ERR_ARG"
    with pytest.raises(comet.CometError) as e:
        comet.transpose(x[1:], [3, 5], [1, 0], out=torch.zeros(15, device="cuda"))
    assert e.value.name == "COMET_ERR_ALIGN"


# ---- the transpose sweep at its full sizes: sampled outputs against the oracle ---------------

SWEEP_PICK = ["r4_f32_p0", "r4_f64_p23", "r6_f32_p5", "r6_f64_p31", "r4_f32_2048MiB", "r6_f64_2048MiB",
              "r6_f32_64MiB"]


@pytest.mark.parametrize("name", SWEEP_PICK)
def test_sweep_case_full_size_sampled(comet, name):
    import math

    import torch
    case = {c[0]: c for c in synth.transpose_sweep_cases()}[name]
    _, rank, es, perm, ext = case
    n = math.prod(ext)
    dt = torch.float32 if es == 4 else torch.float64
    x = synth.torch_uniform(3, 0, n, "cuda", dtype=dt)
    y = comet.transpose(x, ext, perm)
    comet.sync_status()
    sel = np.unique(synth.integers(12, rank, 20000, 0, n - 1).astype(np.int64))
    got = y.view(-1)[torch.from_numpy(sel).cuda()].cpu().numpy()
    host = np.asfortranarray(x.cpu().numpy().reshape(tuple(reversed(ext))).T)
    ref = oracle.transpose_sampled(host, perm, sel)
    assert got.tobytes() == ref.tobytes()
    del x, y


def test_fill(comet):
    import torch
    for dt, val in ((torch.float32, 1.25), (torch.float64, -3.5)):
        for n in (0, 1, 5, 1027, 3_000_001):
            x = torch.full((max(n, 1),), 7.0, dtype=dt, device="cuda")[:n] if n else torch.empty(0, dtype=dt, device="cuda")
            comet.fill(x, val)
            comet.sync_status()
            assert bool((x == val).all())
    y = torch.zeros(10, dtype=torch.float32, device="cuda")
    with pytest.raises(comet.CometError) as e:
        comet.fill(y[1:], 1.0)   # 4-byte offset: not 16-byte aligned
    assert e.value.name == "COMET_ERR_ALIGN"


@pytest.mark.parametrize("extents,perm", [((65539, 32771), (1, 0)), ((5, 32771, 16385), (0, 2, 1))])
def test_above_2_31_elements(comet, extents, perm):
    # more than 2^31 elements: the 64-bit offset variants of the tile and copy kernels.  Each
    # input word holds the low 32 bits of its own linear index, so a sampled check sees any
    # misplaced element.
    import torch
    n = int(np.prod(extents))
    assert n > 2 ** 31
    x = torch.empty(n, dtype=torch.int32, device="cuda")
    step = 1 << 28
    for s in range(0, n, step):
        c = min(n, s + step) - s
        x[s:s + c] = torch.arange(s, s + c, dtype=torch.int64, device="cuda").to(torch.int32)
    xf = x.view(torch.float32)
    out = torch.empty_like(xf)
    comet.transpose(xf, extents, perm, out=out)
    comet.sync_status()
    g = torch.Generator(device="cuda").manual_seed(61)
    j = torch.randint(0, n, (1 << 20,), device="cuda", generator=g, dtype=torch.int64)
    # output index j -> output coordinates (column-major over out extents) -> input linear index
    oext = [extents[p] for p in perm]
    rem, i = j.clone(), torch.zeros_like(j)
    istr = np.cumprod([1] + list(extents[:-1])).tolist()
    for d in range(len(oext)):
        coord = rem % oext[d]
        rem = rem // oext[d]
        i += coord * int(istr[perm[d]])
    got = out.view(torch.int32)[j]
    want = i.to(torch.int32)
    assert bool((got == want).all())
    del x, out
    torch.cuda.empty_cache()
