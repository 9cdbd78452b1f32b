"""GB300 dense tensor contractions in index notation (COMET method, arXiv 2102.06827).

Thin Python binding of the C ABI declared in include/comet.h.  Every step of a contraction
runs in the library's sm_103a kernels; this module only marshals arguments.  PyTorch provides
device memory and streams.  There is no CPU fallback: without the built library every entry
point raises.

Layout convention of the C ABI: column-major in the label order of the expression.  A
column-major tensor with extents (e0, e1, ..., e_{r-1}) is a contiguous torch tensor of shape
(e_{r-1}, ..., e1, e0); ``colmajor_empty`` makes one.  ``einsum`` (in ``autograd``) also
accepts torch's own row-major convention.
"""
from __future__ import annotations

import ctypes
import re
import json

from . import _lib
from ._lib import CometError, F32, F64, PREC_NATIVE, PREC_SPLIT_BF16, PREC_EMU_F64, ORDER_NATURAL, ORDER_PLANNED

__all__ = ["Plan", "BatchedPlan", "transpose", "fill", "sync_status", "colmajor_empty", "CometError",
           "lib", "version", "PREC_NATIVE", "PREC_SPLIT_BF16", "PREC_EMU_F64", "F32", "F64"]


def lib():
    return _lib.load()


def version() -> str:
    return lib().comet_version().decode()


def _dtype_code(dtype) -> int:
    import torch
    if dtype in (torch.float32, "f32", "float32", F32):
        return F32
    if dtype in (torch.float64, "f64", "float64", F64):
        return F64
    raise ValueError(f"unsupported dtype {dtype}")


def _torch_dtype(code: int):
    import torch
    return torch.float32 if code == F32 else torch.float64


def _prec_code(p) -> int:
    if p in ("native", "fp64", PREC_NATIVE, None):
        return PREC_NATIVE
    if p in ("split_bf16", "split", PREC_SPLIT_BF16):
        return PREC_SPLIT_BF16
    if p in ("emu_f64", "emulated_fp64", PREC_EMU_F64):
        return PREC_EMU_F64
    raise ValueError(f"unknown precision {p}")


def _stream_handle(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def colmajor_empty(extents, dtype, device="cuda"):
    """Contiguous torch tensor holding a column-major tensor of the given extents."""
    import torch
    return torch.empty(tuple(reversed([int(e) for e in extents])), dtype=dtype, device=device)


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """comet_plan(): a planned contraction.

    expr     "C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]" (also "+=", "-=", "alpha * ...",
             "sum_{k,c}" and 1..12 operands)
    extents  {label: extent}
    dtype    torch.float32 / torch.float64 (all operands)
    views    optional [(operand, dim, declared, lo, step), ...] (comet_plan_views): dimension
             `dim` (as written) of right-hand operand `operand` (n_in = the left-hand tensor)
             is stored with `declared` indices and the operation takes lo, lo+step, ...
    """

    def __init__(self, expr: str, extents: dict, dtype, precision="native", order="planned",
                 alpha: float = 1.0, workspace_cap: int = 0, form: int = -1, kc: int = 0,
                 timeout_ms: int = 0, debug_flags: int = 0, ksplit: int = 0, host_slices: int = 0,
                 views=None, host_slices_w: int = 0):
        L = lib()
        self.expr = expr
        self.extents = {str(k): int(v) for k, v in extents.items()}
        self.dtype_code = _dtype_code(dtype)
        self.dtype = _torch_dtype(self.dtype_code)
        rhs = expr.split("=", 1)[1] if "=" in expr else ""
        n_ops = len(re.findall(r"[A-Za-z_]\w*\s*[\[(]", rhs))
        self.n_in = n_ops
        ext = (_lib.Extent * max(1, len(self.extents)))(
            *[_lib.Extent(k.encode(), v) for k, v in self.extents.items()])
        dts = (ctypes.c_int * (n_ops + 1))(*([self.dtype_code] * (n_ops + 1)))
        opts = _lib.PlanOpts()
        L.comet_plan_opts_default(ctypes.byref(opts))
        opts.precision = _prec_code(precision)
        opts.order = ORDER_NATURAL if order == "natural" else ORDER_PLANNED
        opts.alpha = alpha
        opts.workspace_cap = workspace_cap
        opts.form = form
        opts.kc = kc
        opts.timeout_ms = timeout_ms
        opts.debug_flags = debug_flags
        opts.ksplit = ksplit
        opts.host_slices = host_slices
        opts.host_slices_w = host_slices_w
        self.precision = opts.precision
        h = ctypes.c_void_p()
        if views:
            vs = (_lib.View * len(views))(*[_lib.View(int(o), int(d), int(n), int(lo), int(st))
                                            for o, d, n, lo, st in views])
            _lib.check(L.comet_plan_views(expr.encode(), ext, len(self.extents), vs, len(views), dts,
                                          n_ops + 1, ctypes.byref(opts), ctypes.byref(h)), "comet_plan_views")
        else:
            _lib.check(L.comet_plan(expr.encode(), ext, len(self.extents), dts, n_ops + 1,
                                    ctypes.byref(opts), ctypes.byref(h)), "comet_plan")
        self._h = h
        ws = ctypes.c_size_t()
        _lib.check(L.comet_plan_workspace(h, ctypes.byref(ws)), "comet_plan_workspace")
        self.workspace_bytes = ws.value
        f = ctypes.c_double()
        _lib.check(L.comet_plan_flops(h, ctypes.byref(f)), "comet_plan_flops")
        self.flops = f.value
        _lib.check(L.comet_plan_flops_natural(h, ctypes.byref(f)), "comet_plan_flops_natural")
        self.flops_natural = f.value
        self.info = self.describe()

    def describe(self) -> dict:
        buf = ctypes.create_string_buffer(1 << 16)
        _lib.check(lib().comet_plan_describe(self._h, buf, len(buf)), "comet_plan_describe")
        return json.loads(buf.value.decode())

    def workspace(self, device="cuda"):
        """A caller-owned workspace buffer of the plan's size (torch allocation)."""
        import torch
        if self.workspace_bytes == 0:
            return None
        return torch.empty(self.workspace_bytes, dtype=torch.uint8, device=device)

    def contract(self, inputs, output, workspace=None, stream=None):
        """comet_contract(): device tensors in, device output tensor written (async)."""
        if len(inputs) != self.n_in:
            raise ValueError(f"{self.n_in} inputs expected")
        arr = (ctypes.c_void_p * self.n_in)(*[t.data_ptr() for t in inputs])
        _lib.check(lib().comet_contract(self._h, arr, _ptr(output), _ptr(workspace),
                                        _stream_handle(stream)), "comet_contract")
        return output

    def contract_host(self, host_inputs, host_output, dev_inputs, dev_output, workspace=None, stream=None):
        """comet_contract_host(): host buffers (numpy arrays or CPU tensors, column-major
        memory) copied in, contracted, copied back; synchronises the stream."""
        def hp(x):
            return ctypes.c_void_p(x.ctypes.data if hasattr(x, "ctypes") else x.data_ptr())
        hin = (ctypes.c_void_p * self.n_in)(*[hp(x).value for x in host_inputs])
        din = (ctypes.c_void_p * self.n_in)(*[t.data_ptr() for t in dev_inputs])
        _lib.check(lib().comet_contract_host(self._h, hin, hp(host_output), din, _ptr(dev_output),
                                             _ptr(workspace), _stream_handle(stream)),
                   "comet_contract_host")
        return host_output

    def contract_host_n(self, host_inputs, host_outputs, dev_inputs, dev_output, workspace=None, stream=None):
        """comet_contract_host_n(): len(host_outputs) evaluations from host buffers, call t taking
        host_inputs[t] (a list of the plan's inputs) and writing host_outputs[t], pipelined
        through one set of device buffers; synchronises the stream."""
        def hp(x):
            return x.ctypes.data if hasattr(x, "ctypes") else x.data_ptr()
        n = len(host_outputs)
        if len(host_inputs) != n or any(len(x) != self.n_in for x in host_inputs):
            raise ValueError("host_inputs: one list of the plan's inputs per output")
        hin = (ctypes.c_void_p * (n * self.n_in))(*[hp(x) for xs in host_inputs for x in xs])
        hout = (ctypes.c_void_p * n)(*[hp(x) for x in host_outputs])
        din = (ctypes.c_void_p * self.n_in)(*[t.data_ptr() for t in dev_inputs])
        _lib.check(lib().comet_contract_host_n(self._h, n, hin, hout, din, _ptr(dev_output), _ptr(workspace),
                                               _stream_handle(stream)),
                   "comet_contract_host_n")
        return host_outputs

    def close(self):
        if getattr(self, "_h", None):
            lib().comet_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchedPlan:
    """comet_plan_batched(): many blocks of one two-operand expression, uneven extents.

    label_names  the labels, in the column order of ``extents``
    extents      integer array n_blocks x n_labels
    """

    def __init__(self, expr: str, label_names, extents, dtype, precision="native", tile: int = -1,
                 timeout_ms: int = 0, debug_flags: int = 0):
        import numpy as np
        L = lib()
        self.expr = expr
        ext = np.ascontiguousarray(np.asarray(extents, dtype=np.int64))
        self.n_blocks, n_labels = ext.shape
        self.dtype_code = _dtype_code(dtype)
        self.dtype = _torch_dtype(self.dtype_code)
        names = (ctypes.c_char_p * n_labels)(*[str(l).encode() for l in label_names])
        dts = (ctypes.c_int * 3)(*([self.dtype_code] * 3))
        opts = _lib.PlanOpts()
        L.comet_plan_opts_default(ctypes.byref(opts))
        opts.precision = _prec_code(precision)
        opts.timeout_ms = timeout_ms
        opts.debug_flags = debug_flags
        h = ctypes.c_void_p()
        _lib.check(L.comet_plan_batched(expr.encode(), self.n_blocks, names, n_labels,
                                        ext.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), dts, 3,
                                        ctypes.byref(opts), tile, ctypes.byref(h)), "comet_plan_batched")
        self._h = h
        ws = ctypes.c_size_t()
        _lib.check(L.comet_plan_workspace(h, ctypes.byref(ws)), "comet_plan_workspace")
        self.workspace_bytes = ws.value
        f = ctypes.c_double()
        _lib.check(L.comet_plan_flops(h, ctypes.byref(f)), "comet_plan_flops")
        self.flops = f.value

    def describe(self) -> dict:
        buf = ctypes.create_string_buffer(1 << 14)
        _lib.check(lib().comet_plan_describe(self._h, buf, len(buf)), "comet_plan_describe")
        return json.loads(buf.value.decode())

    def num_tiles(self) -> int:
        return lib().comet_batched_num_tiles(self._h)

    def set_tile(self, cfg: int):
        _lib.check(lib().comet_batched_set_tile(self._h, cfg), "comet_batched_set_tile")

    def workspace(self, device="cuda"):
        import torch
        return torch.empty(self.workspace_bytes, dtype=torch.uint8, device=device)

    def prepare(self, workspace, stream=None):
        """comet_batched_prepare(): upload the block descriptors (once, before capture)."""
        _lib.check(lib().comet_batched_prepare(self._h, _ptr(workspace), _stream_handle(stream)),
                   "comet_batched_prepare")

    def contract(self, block_inputs, result, workspace, mode: int = 0, key: int = 1, stream=None):
        """comet_contract_batched(): block_inputs is a device int64 tensor of 2*n_blocks
        pointers; result holds 2*n_blocks doubles (mode 0) or n_blocks output pointers (mode 1)."""
        _lib.check(lib().comet_contract_batched(self._h, _ptr(block_inputs), mode, _ptr(result), key,
                                                _ptr(workspace), _stream_handle(stream)),
                   "comet_contract_batched")

    def autotune(self, block_inputs, result, workspace, sample_blocks: int = 0, stream=None):
        """comet_batched_autotune(): (ms per configuration, chosen configuration)."""
        n = self.num_tiles()
        ms = (ctypes.c_double * n)()
        best = ctypes.c_int()
        _lib.check(lib().comet_batched_autotune(self._h, _ptr(block_inputs), _ptr(result), _ptr(workspace),
                                                sample_blocks, _stream_handle(stream), ms, n,
                                                ctypes.byref(best)), "comet_batched_autotune")
        return [ms[i] for i in range(n)], best.value

    def close(self):
        if getattr(self, "_h", None):
            lib().comet_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TriplesPlan:
    """comet_plan_triples(): fused accumulation of permuted terms into six-index blocks and the
    block energies E_b = sum T_b^2 / D_b (see include/comet.h).

    terms        expressions "T[a,b,c,i,j,k] = [alpha *] X[d,a,b,i] * Y[c,d,j,k]" (same T)
    label_names  every label, the columns of ``extents``
    extents      n_blocks x n_labels integers
    signs        six +1 / -1, the sign of each T label's eps in D
    """

    def __init__(self, terms, label_names, extents, signs, dtype):
        import numpy as np
        L = lib()
        ext = np.ascontiguousarray(np.asarray(extents, dtype=np.int64))
        self.n_blocks, n_labels = ext.shape
        self.n_terms = len(terms)
        self.dtype = _torch_dtype(_dtype_code(dtype))
        tv = (ctypes.c_char_p * len(terms))(*[t.encode() for t in terms])
        nv = (ctypes.c_char_p * n_labels)(*[n.encode() for n in label_names])
        sv = (ctypes.c_int * 6)(*[int(x) for x in signs])
        self._ext = ext
        h = ctypes.c_void_p()
        _lib.check(L.comet_plan_triples(tv, len(terms), nv, n_labels, self.n_blocks,
                                        ext.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), sv,
                                        _dtype_code(dtype), ctypes.byref(h)), "comet_plan_triples")
        self._h = h
        ws = ctypes.c_size_t()
        _lib.check(L.comet_plan_workspace(h, ctypes.byref(ws)), "comet_plan_workspace")
        self.workspace_bytes = ws.value
        f = ctypes.c_double()
        _lib.check(L.comet_plan_flops(h, ctypes.byref(f)), "comet_plan_flops")
        self.flops = f.value
        self.info = self.describe()

    def describe(self) -> dict:
        buf = ctypes.create_string_buffer(1 << 16)
        _lib.check(lib().comet_plan_describe(self._h, buf, len(buf)), "comet_plan_describe")
        return json.loads(buf.value.decode())

    def workspace(self, device="cuda"):
        import torch
        return torch.empty(max(16, self.workspace_bytes), dtype=torch.uint8, device=device)

    def prepare(self, workspace, stream=None):
        _lib.check(lib().comet_triples_prepare(self._h, _ptr(workspace), _stream_handle(stream)),
                   "comet_triples_prepare")

    def energy(self, operand_ptrs, eps_ptrs, energies, workspace, stream=None):
        """operand_ptrs: device int64 tensor of n_blocks*n_terms*2 pointers (X, Y per term);
        eps_ptrs: device int64 tensor of n_blocks*6 pointers; energies: device float64[n_blocks]."""
        _lib.check(lib().comet_triples_energy(self._h, _ptr(operand_ptrs), _ptr(eps_ptrs), _ptr(energies),
                                              _ptr(workspace), _stream_handle(stream)), "comet_triples_energy")
        return energies

    def close(self):
        if getattr(self, "_h", None):
            lib().comet_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def transpose(x, extents, perm, out=None, stream=None):
    """comet_transpose(): bit-exact permutation of a column-major tensor.

    out.extent[d] = extents[perm[d]]; returns ``out`` (allocated column-major if None)."""
    import torch
    rank = len(extents)
    if out is None:
        out = colmajor_empty([extents[p] for p in perm], x.dtype, x.device)
    ext = (ctypes.c_int64 * rank)(*[int(e) for e in extents])
    pm = (ctypes.c_int * rank)(*[int(p) for p in perm])
    code = F32 if x.dtype == torch.float32 else F64
    _lib.check(lib().comet_transpose(rank, ext, pm, code, _ptr(x), _ptr(out), _stream_handle(stream)),
               "comet_transpose")
    return out


def fill(x, value, stream=None):
    """comet_fill(): every element of the dense device tensor ``x`` set to ``value``."""
    import torch
    code = F32 if x.dtype == torch.float32 else F64
    _lib.check(lib().comet_fill(_ptr(x), int(x.numel()), float(value), code, _stream_handle(stream)), "comet_fill")
    return x


def profile_enable(on: bool = True):
    """comet_profile_enable(): bracket every library kernel launch with CUDA events."""
    _lib.check(lib().comet_profile_enable(1 if on else 0), "comet_profile_enable")


def profile_read() -> dict:
    """comet_profile_read(): {kernel kind: (launches, total device ms)} since the last read."""
    stats = (_lib.KernelStat * 16)()
    n = ctypes.c_int()
    _lib.check(lib().comet_profile_read(stats, 16, ctypes.byref(n)), "comet_profile_read")
    return {stats[i].name.decode(): (int(stats[i].launches), float(stats[i].total_ms))
            for i in range(min(n.value, 16))}


def sync_status(stream=None):
    """comet_sync_status(): synchronise and surface a device-side timeout."""
    _lib.check(lib().comet_sync_status(_stream_handle(stream)), "comet_sync_status")


FP64_PROBES = {0: "dfma", 1: "dmma_m8n8k4", 2: "dmma_m16n8k4", 3: "dmma_m16n8k16"}


def probe_fp64(kind: int, iters: int, sink, stream=None) -> float:
    """comet_probe_fp64(): launches one FP64 throughput probe kernel (``FP64_PROBES[kind]``) on
    the stream and returns the flops it performs; the caller times the launch."""
    f = ctypes.c_double()
    _lib.check(lib().comet_probe_fp64(int(kind), int(iters), ctypes.byref(f), _ptr(sink),
                                      _stream_handle(stream)), "comet_probe_fp64")
    return f.value
