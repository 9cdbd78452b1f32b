"""CPU FP64 oracle — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline arm of ``bench.py`` may
import this package.  It shares no code with the GPU library: its own expression parser
(below), its own C loops (``oracle.c``), no kernels, no planner.

Arrays are numpy, column-major: an operand written ``A[k,a,c,i]`` is a Fortran-ordered array
of shape ``(ext[k], ext[a], ext[c], ext[i])``.

Functions (each follows the paper's definition it names):
  einsum           Section 2: out = alpha * sum over non-output labels of the product
  abs_einsum       the same with |x|: the scale sum |a||b| of the componentwise error bound
  einsum_sampled   einsum at a list of output linear indices only
  transpose        Section 6 "Transpose optimization": a pure permutation, as a bit move
  transpose_sampled
  triples_reduce   the reduction s = sum T*W, q = sum T^2 of one triples block (a reading:
                   the 6-D triples outputs are consumed in place, not stored)
  grad_exprs       the adjoint expressions of a contraction (each is again a contraction)
  triples_energy   one block of the fused accumulation: T = sum of permuted contributions
                   (each a contraction, Section 2), E = sum T^2 / D with D the signed sum of
                   per-label orbital-energy vectors (the CCSD(T) pattern the paper's Section 3
                   cites: a 6-D output from two 4-D inputs, several terms per block)
"""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain gcc + OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        i64p = ctypes.POINTER(ctypes.c_int64)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_einsum.argtypes = [ctypes.c_int, i64p, ctypes.c_int, ip, ip,
                                    ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ip,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int64, i64p, ctypes.c_void_p]
        L.oracle_transpose.argtypes = [ctypes.c_int, i64p, ip, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int64, i64p]
        L.oracle_triples_reduce.argtypes = [i64p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]
        L.oracle_triples_factor.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        L.oracle_triples_factor.restype = ctypes.c_double
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_fmix32.argtypes = [ctypes.c_uint32]
        L.oracle_fmix32.restype = ctypes.c_uint32
        _lib = L
    return _lib


def threads() -> int:
    return lib().oracle_threads()


# ---------------------------------------------------------------------------------------------
# Expression parser (the paper's operation grammar, Fig. 2b: lhs =|+=|-= [alpha *] T * T ...)
# ---------------------------------------------------------------------------------------------

_TENSOR = re.compile(r"([A-Za-z_][A-Za-z0-9_]*)\s*[\[(]\s*([^\])]*)[\])]")


def parse(expr: str):
    """Returns (out_name, out_labels, op, alpha, [(name, labels), ...]).

    op is "=", "+=" or "-=".  An optional "sum_{k,c}" or "sum_{k c}" marker after the
    assignment is accepted and checked against the labels it names.
    """
    m = re.match(r"\s*(.+?)\s*(\+=|-=|=)\s*(.+)$", expr)
    if not m:
        raise ValueError(f"no assignment in {expr!r}")
    lhs, op, rhs = m.groups()
    lt = _TENSOR.fullmatch(lhs.strip())
    if not lt:
        raise ValueError(f"bad left-hand side {lhs!r}")
    out_name = lt.group(1)
    out_labels = [s.strip() for s in lt.group(2).split(",") if s.strip()]
    declared_sum = None
    sm = re.match(r"\s*sum_\{([^}]*)\}\s*(.*)$", rhs)
    if sm:
        declared_sum = [s for s in re.split(r"[,\s]+", sm.group(1)) if s]
        rhs = sm.group(2)
    factors = [f.strip() for f in rhs.split("*")]
    alpha = 1.0
    operands = []
    for f in factors:
        tm = _TENSOR.fullmatch(f)
        if tm:
            operands.append((tm.group(1), [s.strip() for s in tm.group(2).split(",") if s.strip()]))
        else:
            try:
                alpha *= float(f)
            except ValueError:
                raise ValueError(f"bad factor {f!r}") from None
    if not operands:
        raise ValueError("no operand")
    if declared_sum is not None:
        rhs_labels = {l for _, ls in operands for l in ls}
        if set(declared_sum) != rhs_labels - set(out_labels):
            raise ValueError("sum_{...} does not name the summed labels")
    return out_name, out_labels, op, alpha, operands


def _label_ids(out_labels, operands):
    ids = {}
    for _, ls in operands:
        for l in ls:
            ids.setdefault(l, len(ids))
    for l in out_labels:
        if l not in ids:
            raise ValueError(f"output label {l} appears in no operand")
    return ids


def _extents(ids, operands, arrays):
    ext = [None] * len(ids)
    for (name, ls), a in zip(operands, arrays):
        if a.ndim != len(ls):
            raise ValueError(f"{name}: rank {a.ndim} != {len(ls)} labels")
        for l, e in zip(ls, a.shape):
            if ext[ids[l]] is not None and ext[ids[l]] != e:
                raise ValueError(f"label {l}: extents {ext[ids[l]]} and {e}")
            ext[ids[l]] = e
    return ext


def _call(expr, arrays, mode, alpha_override=None, beta=0.0, out=None, sel=None):
    out_name, out_labels, op, alpha, operands = parse(expr)
    if len(arrays) != len(operands):
        raise ValueError(f"{len(operands)} operands in the expression, {len(arrays)} given")
    if alpha_override is not None:
        alpha = alpha_override
    if op == "+=":
        beta = 1.0
    elif op == "-=":
        alpha, beta = -alpha, 1.0
    ids = _label_ids(out_labels, operands)
    ext = _extents(ids, operands, arrays)
    xs = [np.asfortranarray(np.asarray(a, dtype=np.float64)) for a in arrays]
    out_shape = tuple(ext[ids[l]] for l in out_labels)
    n_in = len(xs)
    ext_c = (ctypes.c_int64 * len(ext))(*ext)
    ranks = (ctypes.c_int * n_in)(*[len(ls) for _, ls in operands])
    flat = [ids[l] for _, ls in operands for l in ls]
    labs = (ctypes.c_int * max(1, len(flat)))(*flat)
    ptrs = (ctypes.c_void_p * n_in)(*[x.ctypes.data for x in xs])
    out_lab = (ctypes.c_int * max(1, len(out_labels)))(*[ids[l] for l in out_labels])
    if sel is None:
        if out is None or beta == 0.0:
            res = np.zeros(out_shape, dtype=np.float64, order="F")
            if out is not None:
                res[...] = out
        else:
            res = np.asfortranarray(np.array(out, dtype=np.float64))
        n_sel, sel_p = 0, None
    else:
        sel = np.ascontiguousarray(np.asarray(sel, dtype=np.int64))
        res = np.zeros(sel.shape[0], dtype=np.float64)
        n_sel = sel.shape[0]
        sel_p = sel.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    rc = lib().oracle_einsum(len(ext), ext_c, n_in, ranks, labs, ptrs, len(out_labels), out_lab,
                             float(alpha), float(beta), mode, n_sel, sel_p,
                             ctypes.c_void_p(res.ctypes.data))
    if rc != 0:
        raise ValueError(f"oracle_einsum rejected the request ({rc})")
    return res


def einsum(expr, *arrays, alpha=None, out=None):
    """Section 2 definition; ``+=``/``-=`` accumulate into ``out`` (beta = 1)."""
    return _call(expr, arrays, 0, alpha_override=alpha, out=out)


def abs_einsum(expr, *arrays):
    """sum over non-output labels of the product of |operands| (alpha and op ignored)."""
    return _call(expr, arrays, 1, alpha_override=1.0)


def einsum_sampled(expr, *arrays, sel, alpha=None):
    """alpha * sum for the output elements whose column-major linear indices are in ``sel``."""
    return _call(expr, arrays, 0, alpha_override=alpha, sel=sel)


def abs_einsum_sampled(expr, *arrays, sel):
    return _call(expr, arrays, 1, alpha_override=1.0, sel=sel)


def transpose(a: np.ndarray, perm) -> np.ndarray:
    """out.shape[d] = a.shape[perm[d]]; out[j] = a[i] with i[perm[d]] = j[d]; raw bit copy."""
    a = np.asfortranarray(a)
    perm = [int(p) for p in perm]
    ext = (ctypes.c_int64 * a.ndim)(*a.shape)
    pc = (ctypes.c_int * a.ndim)(*perm)
    out = np.empty(tuple(a.shape[p] for p in perm), dtype=a.dtype, order="F")
    rc = lib().oracle_transpose(a.ndim, ext, pc, a.itemsize, ctypes.c_void_p(a.ctypes.data),
                                ctypes.c_void_p(out.ctypes.data), 0, None)
    if rc != 0:
        raise ValueError(f"oracle_transpose rejected the request ({rc})")
    return out


def transpose_sampled(a: np.ndarray, perm, sel) -> np.ndarray:
    """Values of transpose(a, perm) at the output column-major linear indices ``sel``."""
    a = np.asfortranarray(a)
    sel = np.ascontiguousarray(np.asarray(sel, dtype=np.int64))
    ext = (ctypes.c_int64 * a.ndim)(*a.shape)
    pc = (ctypes.c_int * a.ndim)(*[int(p) for p in perm])
    out = np.empty(sel.shape[0], dtype=a.dtype)
    rc = lib().oracle_transpose(a.ndim, ext, pc, a.itemsize, ctypes.c_void_p(a.ctypes.data),
                                ctypes.c_void_p(out.ctypes.data), sel.shape[0],
                                sel.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc != 0:
        raise ValueError(f"oracle_transpose rejected the request ({rc})")
    return out


def fmix32(h: int) -> int:
    return lib().oracle_fmix32(h)


def triples_factor(key: int, block: int, x: int) -> float:
    """h(key, block, x) = (fmix32(key ^ fmix32(block * 0x9E3779B9 + x)) >> 8) * 2^-23 - 1."""
    return lib().oracle_triples_factor(key & 0xFFFFFFFF, block, x & 0xFFFFFFFF)


def triples_reduce(A: np.ndarray, B: np.ndarray, key: int, block: int):
    """(s, q) for T[a,b,c,i,j,k] = sum_d A[d,a,b,i] * B[c,d,j,k]:  s = sum T*W, q = sum T^2,
    W = h(key, block, oA) * h(~key, block, oB) with oA (oB) the part of the element's
    column-major linear index that A's labels a, b, i (B's labels c, j, k) contribute."""
    A = np.asfortranarray(A, dtype=np.float64)
    B = np.asfortranarray(B, dtype=np.float64)
    d, a, b, i = A.shape
    c, d2, j, k = B.shape
    if d2 != d:
        raise ValueError("d extents differ")
    ext = (ctypes.c_int64 * 7)(a, b, c, i, j, k, d)
    s, q = ctypes.c_double(), ctypes.c_double()
    rc = lib().oracle_triples_reduce(ext, ctypes.c_void_p(A.ctypes.data),
                                     ctypes.c_void_p(B.ctypes.data), key, block,
                                     ctypes.byref(s), ctypes.byref(q))
    if rc != 0:
        raise ValueError(f"oracle_triples_reduce failed ({rc})")
    return s.value, q.value


def grad_exprs(expr: str):
    """Adjoint expressions of ``out = prod(operands)``: for each operand X, the gradient of
    <G, out> with respect to X is the contraction of G with every other operand onto X's
    labels.  Returns a list of strings "dX[...] = G[...] * Y[...] * ..." (one per operand),
    operand names replaced by position so that repeated names stay distinct."""
    out_name, out_labels, op, alpha, operands = parse(expr)
    res = []
    g = f"G[{','.join(out_labels)}]"
    for x, (_, lx) in enumerate(operands):
        others = [f"X{y}[{','.join(ly)}]" for y, (_, ly) in enumerate(operands) if y != x]
        pre = "" if alpha == 1.0 else f"{alpha!r} * "
        res.append(f"d{x}[{','.join(lx)}] = {pre}{' * '.join([g] + others)}")
    return res


def triples_energy(terms, operands, eps, signs):
    """One block of the fused triples accumulation, by definition:

        T = sum_p einsum(terms[p], X_p, Y_p)      (each term carries its own alpha)
        D[l_1, ..., l_n] = sum_q signs[q] * eps[q][l_q]   (l_q: the q-th label of T)
        E = sum over every element of T^2 / D

    ``terms`` share the left-hand side (T's labels); ``operands`` = [(X_p, Y_p), ...];
    ``eps`` = one vector per T label, in T's label order.  Returns (E, T)."""
    T = None
    for e, (X, Y) in zip(terms, operands):
        t = einsum(e, X, Y)
        T = t if T is None else T + t
    n = T.ndim
    D = np.zeros(T.shape)
    for q in range(n):
        shape = [1] * n
        shape[q] = T.shape[q]
        D = D + signs[q] * np.asarray(eps[q], dtype=np.float64).reshape(shape)
    return float(np.sum(T * T / D)), T
