"""torch.autograd.Function over planned contractions (the differentiation form).

The backward of a contraction is, for every operand that needs a gradient, the adjoint
contraction that comet_adjoint_expr() writes (the incoming gradient contracted with every
other operand onto that operand's labels).  Each adjoint is planned like any expression, so
the adjoint of a multi-operand chain gets its own operand order and recomputes the
intermediates it needs instead of keeping the forward's intermediates alive.  All arithmetic
runs in the library's kernels; this module only builds arguments and allocates buffers.
"""
from __future__ import annotations

import ctypes
import re

import torch

from . import Plan, _lib, lib

_cache: dict = {}

_TENSOR = re.compile(r"([A-Za-z_]\w*)\s*([\[(])([^\])]*)([\])])")


def _reverse_labels(expr: str) -> str:
    """Row-major (torch) labels -> the column-major order of the C ABI: reverse every list."""
    def rev(m):
        labels = [l.strip() for l in m.group(3).split(",") if l.strip()]
        return f"{m.group(1)}{m.group(2)}{','.join(reversed(labels))}{m.group(4)}"
    return _TENSOR.sub(rev, expr)


def adjoint_expr(expr: str, operand: int) -> str:
    buf = ctypes.create_string_buffer(4096)
    _lib.check(lib().comet_adjoint_expr(expr.encode(), operand, buf, len(buf)), "comet_adjoint_expr")
    return buf.value.decode()


def _plan(expr, ext, dtype, precision, order, workspace_cap):
    key = (expr, tuple(sorted(ext.items())), dtype, precision, order, workspace_cap)
    p = _cache.get(key)
    if p is None:
        p = Plan(expr, ext, dtype, precision=precision, order=order, workspace_cap=workspace_cap)
        _cache[key] = p
    return p


def _labels(expr):
    tensors = _TENSOR.findall(expr)
    out = [l.strip() for l in tensors[0][2].split(",") if l.strip()]
    ins = [[l.strip() for l in t[2].split(",") if l.strip()] for t in tensors[1:]]
    return out, ins


def _run(expr, ext, tensors, precision, order, workspace_cap):
    t0 = tensors[0]
    p = _plan(expr, ext, t0.dtype, precision, order, workspace_cap)
    out_labels, _ = _labels(expr)
    out = torch.empty(tuple(reversed([ext[l] for l in out_labels])), dtype=t0.dtype, device=t0.device)
    p.contract([t.contiguous() for t in tensors], out, p.workspace(t0.device))
    return out


class ContractFunction(torch.autograd.Function):
    """forward(expr, precision, order, workspace_cap, *tensors): column-major expression."""

    @staticmethod
    def forward(ctx, expr, precision, order, workspace_cap, *tensors):
        out_labels, in_labels = _labels(expr)
        ext = {}
        for labels, t in zip(in_labels, tensors):
            if t.dim() != len(labels):
                raise ValueError(f"rank {t.dim()} tensor for {len(labels)} labels")
            for l, e in zip(labels, reversed(t.shape)):
                ext[l] = int(e)
        ctx.expr, ctx.precision, ctx.order, ctx.cap, ctx.ext = expr, precision, order, workspace_cap, ext
        ctx.save_for_backward(*tensors)
        return _run(expr, ext, tensors, precision, order, workspace_cap)

    @staticmethod
    def backward(ctx, grad):
        tensors = ctx.saved_tensors
        grads = []
        for p in range(len(tensors)):
            if not ctx.needs_input_grad[4 + p]:
                grads.append(None)
                continue
            adj = adjoint_expr(ctx.expr, p)
            others = [grad.contiguous()] + [tensors[t] for t in range(len(tensors)) if t != p]
            grads.append(_run(adj, ctx.ext, others, ctx.precision, ctx.order, ctx.cap))
        return (None, None, None, None, *grads)


def einsum(expr: str, *tensors, precision="split_bf16", order="planned", layout="row", workspace_cap=0):
    """Differentiable contraction.  layout "row": torch's convention (tensor.shape[d] is the
    extent of the d-th label); "col": column-major (shape reversed), the C ABI's convention."""
    e = _reverse_labels(expr) if layout == "row" else expr
    return ContractFunction.apply(e, precision, order, workspace_cap, *tensors)
