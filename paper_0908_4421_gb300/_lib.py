"""ctypes declarations of the C ABI in include/imrt.h (argument marshalling only).

The structures mirror the header field by field; the functions keep the C
names. Loading fails loudly when libimrt.so has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libimrt.so")

IMRT_OK, IMRT_EINVAL, IMRT_ENOMEM, IMRT_ECUDA, IMRT_ELINESEARCH = 0, 1, 2, 3, 4
IMRT_ENUMERIC, IMRT_ETIMEOUT, IMRT_ECANCELLED, IMRT_EUNSUPPORTED = 5, 6, 7, 8
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ELINESEARCH", 5: "ENUMERIC",
                6: "ETIMEOUT", 7: "ECANCELLED", 8: "EUNSUPPORTED"}
STOP_NONE, STOP_REL, STOP_MAXITER, STOP_EXACT, STOP_STATIONARY = 0, 1, 2, 3, 4
FP32, FP16, BF16, FP8E4M3 = 0, 1, 2, 3
MODE_GRAPH, MODE_HOST = 0, 1
SOLVER_GRAPH, SOLVER_TEAM = 0, 1

# Every symbol include/imrt.h declares.
EXPORTS = ("imrt_default_options", "plan_create", "plan_set_options", "plan_solve", "plan_dose", "plan_eval",
           "plan_get_x", "plan_get_trace", "plan_info", "plan_cancel", "plan_destroy", "imrt_last_error",
           "imrt_version", "imrt_eval_csr_noalloc", "plan_solve_batch", "plan_set_voxel_targets",
           "imrt_trim_memory", "plan_update")


class imrt_csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("on_device", ctypes.c_int32)]


class imrt_options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("alpha", ctypes.c_double), ("lambda0", ctypes.c_double),
                ("delta", ctypes.c_double), ("max_iter", ctypes.c_int32), ("max_backtracks", ctypes.c_int32),
                ("x_init", ctypes.c_int32), ("precision", ctypes.c_int32), ("k_trials", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("profile", ctypes.c_int32), ("trace", ctypes.c_int32),
                ("polish_iter", ctypes.c_int32), ("kernel_variant", ctypes.c_int32), ("timeout_ms", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("solver", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("polish_switch", ctypes.c_double)]


class imrt_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("stop_reason", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("backtracks", ctypes.c_int32), ("passes", ctypes.c_int32), ("grad_passes", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("polish_iterations", ctypes.c_int32),
                ("objective", ctypes.c_double), ("initial_objective", ctypes.c_double), ("kkt", ctypes.c_double),
                ("rel_change", ctypes.c_double), ("lambda0", ctypes.c_double), ("ms", ctypes.c_double),
                ("fwd_ms", ctypes.c_double), ("bwd_ms", ctypes.c_double), ("fwd_launches", ctypes.c_int32),
                ("bwd_launches", ctypes.c_int32), ("bytes", ctypes.c_int64)]


class imrt_plan_info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("n_structures", ctypes.c_int32),
                ("n_slices", ctypes.c_int32), ("nnz", ctypes.c_int64), ("sell_entries", ctypes.c_int64),
                ("t_entries", ctypes.c_int64), ("fwd_bytes", ctypes.c_int64), ("bwd_bytes", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("fwd_grid", ctypes.c_int32), ("fwd_block", ctypes.c_int32),
                ("bwd_grid", ctypes.c_int32), ("bwd_block", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("k_trials", ctypes.c_int32), ("lambda0_rule", ctypes.c_double), ("x1_scale", ctypes.c_double),
                ("fwd_schedule", ctypes.c_int32), ("fwd_units", ctypes.c_int32)]


_lib: Optional[ctypes.CDLL] = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libimrt.so (built by __graft_entry__.build() / paper_0908_4421_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    lib.imrt_default_options.restype = None
    lib.imrt_default_options.argtypes = [P(imrt_options)]
    lib.plan_create.restype = ctypes.c_int
    lib.plan_create.argtypes = [P(imrt_csr), vp, ctypes.c_int32, vp, vp, P(imrt_options), P(vp)]
    lib.plan_update.restype = ctypes.c_int
    lib.plan_update.argtypes = [vp, P(imrt_csr), vp, ctypes.c_int32, vp, vp]
    lib.plan_set_options.restype = ctypes.c_int
    lib.plan_set_options.argtypes = [vp, P(imrt_options)]
    lib.plan_solve.restype = ctypes.c_int
    lib.plan_solve.argtypes = [vp, vp, P(imrt_result)]
    lib.plan_set_voxel_targets.restype = ctypes.c_int
    lib.plan_set_voxel_targets.argtypes = [vp, vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_int32]
    lib.plan_solve_batch.restype = ctypes.c_int
    lib.plan_solve_batch.argtypes = [vp, ctypes.c_int32, vp, vp, vp]
    lib.plan_dose.restype = ctypes.c_int
    lib.plan_dose.argtypes = [vp, vp, vp]
    lib.plan_eval.restype = ctypes.c_int
    lib.plan_eval.argtypes = [vp, vp, vp, vp, vp]
    lib.plan_get_x.restype = ctypes.c_int
    lib.plan_get_x.argtypes = [vp, vp]
    lib.plan_get_trace.restype = ctypes.c_int
    lib.plan_get_trace.argtypes = [vp, ctypes.c_int32, vp, vp, vp, vp]
    lib.plan_info.restype = ctypes.c_int
    lib.plan_info.argtypes = [vp, P(imrt_plan_info)]
    lib.plan_cancel.restype = ctypes.c_int
    lib.plan_cancel.argtypes = [vp]
    lib.plan_destroy.restype = None
    lib.plan_destroy.argtypes = [vp]
    lib.imrt_last_error.restype = ctypes.c_char_p
    lib.imrt_last_error.argtypes = []
    lib.imrt_version.restype = ctypes.c_char_p
    lib.imrt_version.argtypes = []
    lib.imrt_trim_memory.restype = ctypes.c_int
    lib.imrt_trim_memory.argtypes = [ctypes.c_size_t]
    lib.imrt_eval_csr_noalloc.restype = ctypes.c_int
    lib.imrt_eval_csr_noalloc.argtypes = [P(imrt_csr), vp, ctypes.c_int32, vp, vp, vp, vp, vp, vp]
    _lib = lib
    return lib


class ImrtError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status: int) -> int:
    if status != IMRT_OK:
        raise ImrtError(status, load().imrt_last_error().decode())
    return status
