"""ctypes binding of libpolartrace (include/polartrace.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts torch
tensors to device pointers, allocates the caller-owned workspaces with torch
and maps status codes to exceptions.  There is no CPU fallback: if the
library is missing the import of :func:`lib` fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libpolartrace.so")

PT_FP64, PT_MIXED_FP32, PT_MIXED_TC = 0, 1, 2
STATUS = ["PT_OK", "PT_ERR_ARG", "PT_ERR_WORKSPACE", "PT_ERR_CUDA", "PT_ERR_SINGULAR", "PT_ERR_NOT_CONVERGED",
          "PT_ERR_TIMEOUT", "PT_ERR_NUMERIC"]

# every symbol include/polartrace.h declares
EXPORTS = [
    "pt_layer_partition", "pt_workspace_size", "pt_create", "pt_solve", "pt_solve_host", "pt_apply_matvec",
    "pt_apply_precond", "pt_apply_D_inverse", "pt_apply_R", "pt_rhs", "pt_get_block", "pt_last_solve_stats",
    "pt_destroy", "pt_status_string", "pt_last_error", "pt_rhs_noalloc", "pt_apply", "pt_plr_stats",
    "pt_volume_residual", "pt_set_option", "pt_correction_nparams", "pt_set_correction", "pt_get_correction",
    "pt_correction_scratch_bytes", "pt_correction_forward", "pt_correction_grad", "pt_train_bytes",
    "pt_train_correction", "pt_apply_correction", "pt_last_solve_cycles", "pt_solve_many", "pt_last_solve_relaxed",
    "pt_solve_gs",
]
PT_OPT_LAYER_GROUP = 1
PT_OPT_LEARNED = 2
PT_OPT_LOCAL_SOLVE = 3
PT_OPT_SWEEP = 4
PT_OPT_RELAX = 5
PT_OPT_PRECOND_FP16 = 6
PT_OPT_RESTART = 7


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("nz", C.c_int32), ("npml", C.c_int32), ("L", C.c_int32),
        ("h", C.c_double), ("omega", C.c_double), ("pml_C", C.c_double),
        ("precision", C.c_int32), ("gs_iters", C.c_int32), ("max_sources", C.c_int32), ("max_krylov", C.c_int32),
        ("plr", C.c_int32), ("plr_eps", C.c_double), ("plr_rmax", C.c_int32), ("learned", C.c_int32),
        ("layer_rows", C.POINTER(C.c_int32)),
    ]


class PolarTraceError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{where}: {name}: {detail}")


_lib = None


def lib() -> C.CDLL:
    """Load the library (built by ``paper_1410_5910_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1410_5910_gb300.build`")
    L = C.CDLL(LIB_PATH)
    vp, sz, i32, f64 = C.c_void_p, C.c_size_t, C.c_int32, C.c_double
    P = C.POINTER(Params)
    L.pt_layer_partition.argtypes = [P, C.POINTER(i32)]
    L.pt_workspace_size.argtypes = [P, C.POINTER(sz), C.POINTER(sz), C.POINTER(sz)]
    L.pt_create.argtypes = [P, vp, vp, sz, vp, sz, vp, C.POINTER(vp)]
    L.pt_solve.argtypes = [vp, i32, vp, vp, vp, f64, i32, vp, sz, C.POINTER(i32), C.POINTER(f64)]
    L.pt_solve_gs.argtypes = [vp, i32, vp, vp, vp, f64, i32, vp, sz, C.POINTER(i32), C.POINTER(f64)]
    L.pt_solve_host.argtypes = [vp, i32, vp, vp, f64, i32, vp, sz, C.POINTER(i32), C.POINTER(f64)]
    for name in ("pt_apply_matvec", "pt_apply_D_inverse", "pt_apply_R"):
        getattr(L, name).argtypes = [vp, i32, vp, vp]
    L.pt_apply_precond.argtypes = [vp, i32, vp, vp, vp, sz]
    L.pt_rhs.argtypes = [vp, i32, vp, vp, vp, sz]
    L.pt_rhs_noalloc.argtypes = [vp, i32, vp, vp]
    L.pt_apply.argtypes = [vp, i32, i32, i32, vp, vp, vp, sz]
    L.pt_plr_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(i32)]
    L.pt_volume_residual.argtypes = [vp, i32, vp, vp, C.POINTER(f64), vp, sz]
    L.pt_get_block.argtypes = [vp, i32, i32, i32, vp]
    L.pt_set_option.argtypes = [vp, i32, i32]
    i64, u64 = C.c_int64, C.c_uint64
    L.pt_correction_nparams.argtypes = [C.POINTER(i64)]
    L.pt_set_correction.argtypes = [vp, vp, i64]
    L.pt_get_correction.argtypes = [vp, vp, i64]
    L.pt_correction_scratch_bytes.argtypes = [vp, i32, C.POINTER(sz)]
    L.pt_correction_forward.argtypes = [vp, i32, vp, vp, vp, sz]
    L.pt_correction_grad.argtypes = [vp, i32, vp, vp, C.POINTER(f64), vp, vp, sz]
    L.pt_train_bytes.argtypes = [vp, i32, i32, C.POINTER(sz)]
    L.pt_train_correction.argtypes = [vp, i32, vp, vp, i32, i32, f64, u64, C.POINTER(f64), C.POINTER(f64), vp, sz]
    L.pt_apply_correction.argtypes = [vp, i32, vp, vp, vp, sz]
    L.pt_last_solve_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(i32)]
    L.pt_last_solve_cycles.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
    L.pt_last_solve_relaxed.argtypes = [vp, C.POINTER(i32)]
    L.pt_solve_many.argtypes = [i32, C.POINTER(vp), C.POINTER(i32), C.POINTER(vp), C.POINTER(vp), f64, i32,
                                C.POINTER(vp), C.POINTER(sz), C.POINTER(i32), C.POINTER(f64), C.POINTER(i32)]
    L.pt_destroy.argtypes = [vp]
    L.pt_destroy.restype = None
    L.pt_status_string.argtypes = [i32]
    L.pt_status_string.restype = C.c_char_p
    L.pt_last_error.argtypes = []
    L.pt_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("pt_destroy", "pt_status_string", "pt_last_error"):
            getattr(L, name).restype = i32
    _lib = L
    return L


def check(status: int, where: str, allow=()) -> int:
    if status != 0 and status not in allow:
        raise PolarTraceError(status, where, lib().pt_last_error().decode())
    return status
