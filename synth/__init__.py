"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This module holds no contraction arithmetic: it only turns (seed, tensor id, element index)
into numbers.  The generator is counter based, so any element can be produced on its own and
the bits do not depend on numpy, torch or libm versions.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014).  The value for counter ``n`` of a stream with key ``k`` is the
SplitMix64 output function applied to ``k + (n + 1) * GAMMA``; the stream key itself is the
output function applied to ``seed * GAMMA + tensor_id``.

Layout convention: tensors are column-major (first label fastest).  As numpy arrays they are
Fortran-ordered with ``shape[d]`` = extent of the d-th label; element ``n`` of the stream is
the element with column-major linear index ``n``.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1
_CHUNK = 1 << 22


def mix64_int(z: int) -> int:
    """SplitMix64 output function on one Python int (mod 2**64)."""
    z &= _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def stream_key(seed: int, tensor_id: int) -> int:
    return mix64_int((seed * GAMMA + tensor_id) & _MASK)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        return z ^ (z >> np.uint64(31))


def raw_bits(seed: int, tensor_id: int, start: int, count: int) -> np.ndarray:
    """uint64 stream values for counters start .. start+count-1."""
    key = np.uint64(stream_key(seed, tensor_id))
    n = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64_np(key + n * np.uint64(GAMMA))


def _fill(count: int, fn) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    for s in range(0, count, _CHUNK):
        e = min(count, s + _CHUNK)
        out[s:e] = fn(s, e - s)
    return out


def uniform(seed: int, tensor_id: int, count: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """float64 values in [lo, hi): top 53 bits of each stream value as a fraction."""
    def f(s, c):
        u = (raw_bits(seed, tensor_id, s, c) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        return lo + (hi - lo) * u
    return _fill(count, f)


def normal(seed: int, tensor_id: int, count: int, std: float = 1.0) -> np.ndarray:
    """float64 normal(0, std) by the Box-Muller transform on counter pairs (2n, 2n+1)."""
    def f(s, c):
        bits = raw_bits(seed, tensor_id, 2 * s, 2 * c)
        u = ((bits >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53  # (0, 1)
        u1, u2 = u[0::2], u[1::2]
        return std * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return _fill(count, f)


def integers(seed: int, tensor_id: int, count: int, lo: int, hi: int) -> np.ndarray:
    """float64 integers uniform in [lo, hi] (inclusive); exact in every float format used."""
    span = hi - lo + 1
    def f(s, c):
        return (raw_bits(seed, tensor_id, s, c) % np.uint64(span)).astype(np.float64) + lo
    return _fill(count, f)


def tensor(extents, seed: int, tensor_id: int, kind: str = "uniform", dtype=np.float64,
           scale: float = 1.0, **kw) -> np.ndarray:
    """Column-major (Fortran-ordered) tensor of the given extents.

    kind: "uniform" ([-1,1) times scale), "normal" (std = scale), "int" (integers in
    [kw lo, kw hi]), "ones".
    """
    extents = tuple(int(e) for e in extents)
    count = int(np.prod(extents, dtype=np.int64)) if extents else 1
    if kind == "uniform":
        v = uniform(seed, tensor_id, count) * scale
    elif kind == "normal":
        v = normal(seed, tensor_id, count, std=scale)
    elif kind == "int":
        v = integers(seed, tensor_id, count, kw.get("lo", -4), kw.get("hi", 4))
    elif kind == "ones":
        v = np.ones(count)
    else:
        raise ValueError(kind)
    return np.asfortranarray(v.astype(dtype).reshape(extents, order="F"))


def uniform_extents(seed: int, tensor_id: int, count: int, lo: int, hi: int) -> np.ndarray:
    """int64 extents uniform in [lo, hi] (inclusive)."""
    return integers(seed, tensor_id, count, lo, hi).astype(np.int64)


# --- the same generator on a torch device (for inputs too large to build on the host) ----------

def torch_uniform(seed: int, tensor_id: int, count: int, device, dtype=None, scale: float = 1.0):
    """Bit-identical to ``uniform(...) * scale`` but built on ``device`` with int64 arithmetic
    (two's-complement wraparound; logical shifts emulated with masks)."""
    import torch
    key = stream_key(seed, tensor_id)
    key_s = key - (1 << 64) if key >= (1 << 63) else key
    out = torch.empty(count, dtype=torch.float64, device=device)
    g = GAMMA - (1 << 64)
    m1 = _M1 - (1 << 64)
    m2 = _M2 - (1 << 64)

    def lsr(z, s):
        return (z >> s) & ((1 << (64 - s)) - 1)

    step = 1 << 24
    for s in range(0, count, step):
        c = min(count, s + step) - s
        n = torch.arange(s + 1, s + c + 1, dtype=torch.int64, device=device)
        z = n * g + key_s
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        z = z ^ lsr(z, 31)
        u = lsr(z, 11).to(torch.float64) * 2.0 ** -53
        out[s:s + c] = (-1.0 + 2.0 * u) * scale
    return out if dtype is None else out.to(dtype)


# --- the transpose sweep: rank-4 (all 24 permutations) and rank-6 (32 seeded permutations),
# FP32 and FP64, 64 MiB to 2 GiB, extents in 8..256 -------------------------------------------

class _Stream:
    """Sequential draws from one SplitMix64 stream (for shape and permutation choices)."""

    def __init__(self, seed, tensor_id):
        self.key = stream_key(seed, tensor_id)
        self.n = 0

    def next(self) -> int:
        self.n += 1
        return mix64_int(self.key + self.n * GAMMA)

    def uniform(self) -> float:
        return (self.next() >> 11) * 2.0 ** -53

    def below(self, k: int) -> int:
        return self.next() % k


def transpose_sweep_cases(max_bytes: int = 2 << 30, min_bytes: int = 64 << 20):
    """[(name, rank, elem_bytes, perm, extents)].  Per (rank, dtype, perm): target bytes
    log-uniform in [min_bytes, max_bytes], rank-1 extents log-uniform in [8, 256], the last
    extent fixed by the target (redrawn while outside [8, 256]).  Seeds: 1000*rank + 10*dtype +
    perm index.  Plus fixed shapes of exactly 64 MiB and 2 GiB per rank and dtype."""
    import itertools
    import math
    cases = []
    perms4 = list(itertools.permutations(range(4)))
    ps = _Stream(6, 0)
    perms6 = []
    while len(perms6) < 32:
        p = list(range(6))
        for i in range(5, 0, -1):          # Fisher-Yates with the stream
            j = ps.below(i + 1)
            p[i], p[j] = p[j], p[i]
        if tuple(p) not in perms6 and tuple(p) != tuple(range(6)):
            perms6.append(tuple(p))
    for rank, perms in ((4, perms4), (6, perms6)):
        for dt, es in ((0, 4), (1, 8)):
            for pi, perm in enumerate(perms):
                st = _Stream(1000 * rank + 10 * dt + pi, 1)
                for _ in range(1000):
                    target = math.exp(math.log(min_bytes) + st.uniform() * (math.log(max_bytes) - math.log(min_bytes)))
                    ext = [int(round(math.exp(math.log(8) + st.uniform() * (math.log(256) - math.log(8)))))
                           for _ in range(rank - 1)]
                    last = int(round(target / (es * math.prod(ext))))
                    if 8 <= last <= 256:
                        ext.append(last)
                        break
                else:
                    raise RuntimeError("no shape found")
                cases.append((f"r{rank}_{'f32' if es == 4 else 'f64'}_p{pi}", rank, es, tuple(perm), tuple(ext)))
    fixed = {4: {64 << 20: [(64, 128, 128, 16), (32, 128, 128, 16)],
                 2 << 30: [(128, 256, 128, 128), (64, 256, 128, 128)]},
             6: {64 << 20: [(16, 16, 16, 16, 16, 16), (16, 16, 16, 16, 16, 8)],
                 2 << 30: [(32, 32, 32, 32, 32, 16), (32, 32, 32, 32, 32, 8)]}}
    for rank in (4, 6):
        for size, shapes in fixed[rank].items():
            if size > max_bytes:
                continue
            for es, shape in zip((4, 8), shapes):
                perm = tuple(reversed(range(rank))) if rank == 4 else (1, 3, 5, 0, 2, 4)
                cases.append((f"r{rank}_{'f32' if es == 4 else 'f64'}_{size >> 20}MiB", rank, es, perm, shape))
    return cases


def torch_normal(seed: int, tensor_id: int, count: int, device, dtype=None, std: float = 1.0):
    """normal(0, std) on ``device`` by the Box-Muller transform of ``normal`` (same counters and
    formula; values agree with the host version to within a few units in the last place of the
    device's log/sqrt/cos)."""
    import torch
    key = stream_key(seed, tensor_id)
    key_s = key - (1 << 64) if key >= (1 << 63) else key
    g = GAMMA - (1 << 64)
    m1 = _M1 - (1 << 64)
    m2 = _M2 - (1 << 64)

    def lsr(z, s):
        return (z >> s) & ((1 << (64 - s)) - 1)

    def mix(n):
        z = n * g + key_s
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        return z ^ lsr(z, 31)

    out = torch.empty(count, dtype=torch.float64, device=device)
    step = 1 << 23
    for s in range(0, count, step):
        c = min(count, s + step) - s
        n = torch.arange(2 * s + 1, 2 * (s + c) + 1, dtype=torch.int64, device=device)
        u = (lsr(mix(n), 11).to(torch.float64) + 0.5) * 2.0 ** -53
        u1, u2 = u[0::2], u[1::2]
        out[s:s + c] = std * torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
    return out if dtype is None else out.to(dtype)


def triples_blocks(n_blocks: int = 4096, lo: int = 8, hi: int = 32, seed: int = 3):
    """Extents of the batched triples workload: an n_blocks x 7 table over the labels
    (a, b, c, i, j, k, d), each uniform in [lo, hi], drawn from the seed."""
    return integers(seed, 0, n_blocks * 7, lo, hi).astype(np.int64).reshape(n_blocks, 7)


def normal_range(seed: int, tensor_id: int, start: int, count: int, std: float = 1.0) -> np.ndarray:
    """Elements start .. start+count-1 of the ``normal`` stream."""
    bits = raw_bits(seed, tensor_id, 2 * start, 2 * count)
    u = ((bits >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    return std * np.sqrt(-2.0 * np.log(u[0::2])) * np.cos(2.0 * np.pi * u[1::2])
