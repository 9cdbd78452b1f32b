"""ctypes declarations of the C ABI in include/comet.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcomet.so")

COMET_OK = 0
STATUS = {
    0: "COMET_OK", 1: "COMET_ERR_PARSE", 2: "COMET_ERR_LABEL", 3: "COMET_ERR_SHAPE",
    4: "COMET_ERR_DTYPE", 5: "COMET_ERR_UNSUPPORTED", 6: "COMET_ERR_ALIGN", 7: "COMET_ERR_NULL",
    8: "COMET_ERR_WORKSPACE", 9: "COMET_ERR_CUDA", 10: "COMET_ERR_TIMEOUT",
    11: "COMET_ERR_INTERNAL", 12: "COMET_ERR_ARG", 13: "COMET_ERR_BOUNDS",
}
F32, F64 = 0, 1
PREC_NATIVE, PREC_SPLIT_BF16, PREC_EMU_F64 = 0, 1, 2
ORDER_PLANNED, ORDER_NATURAL = 0, 1

# every symbol include/comet.h declares (checked by the CPU test suite)
EXPORTS = [
    "comet_plan_opts_default", "comet_plan", "comet_plan_views", "comet_plan_workspace", "comet_plan_flops",
    "comet_plan_flops_natural", "comet_plan_describe", "comet_adjoint_expr", "comet_contract", "comet_contract_noalloc", "comet_contract_host",
    "comet_contract_host_n",
    "comet_transpose", "comet_fill", "comet_plan_batched", "comet_batched_num_tiles", "comet_batched_set_tile",
    "comet_batched_prepare", "comet_contract_batched", "comet_batched_autotune",
    "comet_plan_triples", "comet_triples_prepare", "comet_triples_energy",
    "comet_profile_enable", "comet_profile_read", "comet_probe_fp64", "comet_sync_status", "comet_plan_destroy", "comet_status_string", "comet_last_error_message",
    "comet_version",
]


class CometError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        self.name = STATUS.get(code, str(code))
        super().__init__(f"{where}: {self.name}" + (f" ({detail})" if detail else ""))


class Extent(ctypes.Structure):
    _fields_ = [("label", ctypes.c_char_p), ("extent", ctypes.c_int64)]


class View(ctypes.Structure):
    _fields_ = [("operand", ctypes.c_int), ("dim", ctypes.c_int), ("declared", ctypes.c_int64),
                ("lo", ctypes.c_int64), ("step", ctypes.c_int64)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class PlanOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("order", ctypes.c_int), ("alpha", ctypes.c_double),
                ("workspace_cap", ctypes.c_size_t), ("form", ctypes.c_int), ("kc", ctypes.c_int64),
                ("timeout_ms", ctypes.c_int64), ("debug_flags", ctypes.c_int),
                ("ksplit", ctypes.c_int), ("host_slices", ctypes.c_int), ("host_slices_w", ctypes.c_int)]


_lib = None


def load():
    """Loads the in-tree libcomet.so (or the library COMET_LIBRARY names, e.g. the debug build
    libcomet_debug.so); raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("COMET_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{os.path.basename(path)} is not built ({path}); run __graft_entry__.build() "
                          "or python paper_2102_06827_gb300/build.py")
    L = ctypes.CDLL(path)
    vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
    L.comet_plan_opts_default.argtypes = [ctypes.POINTER(PlanOpts)]
    L.comet_plan_opts_default.restype = None
    L.comet_plan.argtypes = [ctypes.c_char_p, ctypes.POINTER(Extent), ctypes.c_int,
                             ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(PlanOpts),
                             ctypes.POINTER(vp)]
    L.comet_plan_views.argtypes = [ctypes.c_char_p, ctypes.POINTER(Extent), ctypes.c_int,
                                   ctypes.POINTER(View), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.c_int, ctypes.POINTER(PlanOpts), ctypes.POINTER(vp)]
    L.comet_adjoint_expr.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t]
    L.comet_plan_workspace.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.comet_plan_flops.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.comet_plan_flops_natural.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.comet_plan_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    L.comet_contract.argtypes = [vp, ctypes.POINTER(vp), vp, vp, vp]
    L.comet_contract_noalloc.argtypes = [vp, ctypes.POINTER(vp), vp, vp]
    L.comet_contract_host.argtypes = [vp, ctypes.POINTER(vp), vp, ctypes.POINTER(vp), vp, vp, vp]
    L.comet_contract_host_n.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                        ctypes.POINTER(vp), vp, vp, vp]
    L.comet_transpose.argtypes = [ctypes.c_int, i64p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                  vp, vp, vp]
    L.comet_fill.argtypes = [vp, ctypes.c_int64, ctypes.c_double, ctypes.c_int, vp]
    L.comet_plan_batched.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                     ctypes.c_int, i64p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                     ctypes.POINTER(PlanOpts), ctypes.c_int, ctypes.POINTER(vp)]
    L.comet_batched_num_tiles.argtypes = [vp]
    L.comet_batched_num_tiles.restype = ctypes.c_int
    L.comet_batched_set_tile.argtypes = [vp, ctypes.c_int]
    L.comet_batched_prepare.argtypes = [vp, vp, vp]
    L.comet_contract_batched.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_uint32, vp, vp]
    L.comet_batched_autotune.argtypes = [vp, vp, vp, vp, ctypes.c_int, vp,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]
    L.comet_plan_triples.argtypes = [ctypes.POINTER(ctypes.c_char_p), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_char_p), ctypes.c_int, ctypes.c_int, i64p,
                                     ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(vp)]
    L.comet_triples_prepare.argtypes = [vp, vp, vp]
    L.comet_triples_energy.argtypes = [vp, vp, vp, vp, vp, vp]
    L.comet_profile_enable.argtypes = [ctypes.c_int]
    L.comet_profile_read.argtypes = [ctypes.POINTER(KernelStat), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.comet_probe_fp64.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), vp, vp]
    L.comet_sync_status.argtypes = [vp]
    L.comet_plan_destroy.argtypes = [vp]
    L.comet_plan_destroy.restype = None
    L.comet_status_string.argtypes = [ctypes.c_int]
    L.comet_status_string.restype = ctypes.c_char_p
    L.comet_last_error_message.argtypes = []
    L.comet_last_error_message.restype = ctypes.c_char_p
    L.comet_version.argtypes = []
    L.comet_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("comet_plan_opts_default", "comet_plan_destroy", "comet_status_string",
                        "comet_last_error_message", "comet_version", "comet_batched_num_tiles"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(code: int, where: str):
    if code != COMET_OK:
        detail = load().comet_last_error_message().decode(errors="replace")
        raise CometError(code, where, detail)
