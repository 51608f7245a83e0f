"""Python binding of the C ABI: a thin ``Plan`` wrapper (argument marshalling only).

Every step of the solve runs in libimrt's CUDA kernels; this module converts
numpy arrays or torch CUDA tensors into pointers, fills the option structure,
and turns status codes into exceptions. torch is used only for device buffers
and the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional

import numpy as np

from . import _lib as L


@dataclasses.dataclass
class Options:
    """Mirror of imrt_options (defaults = imrt_default_options)."""

    eps: float = 1e-4
    alpha: float = 2.0
    lambda0: float = 0.0
    delta: float = 1e-6
    max_iter: int = 200
    max_backtracks: int = 50
    x_init: int = 0
    precision: int = L.FP32
    k_trials: int = 1
    mode: int = L.MODE_GRAPH
    profile: int = 0
    trace: int = 0
    polish_iter: int = 20
    kernel_variant: int = 0  # forward pass: 0 warp streaming, CTA-local schedule; 1 bulk-copy (TMA); 2 global schedule
    timeout_ms: float = 0.0
    stream: int = 0  # cudaStream_t as an integer; 0 = legacy default stream
    solver: int = L.SOLVER_GRAPH  # SOLVER_TEAM: the persistent multi-plan kernel
    reserved: int = 0
    polish_switch: float = 0.0  # reduced precision: hand over to the FP32 polish below this relative change

    def to_c(self) -> L.imrt_options:
        o = L.imrt_options()
        for f in dataclasses.fields(self):
            setattr(o, f.name, getattr(self, f.name))
        return o


@dataclasses.dataclass
class Result:
    status: int
    stop_reason: int
    iterations: int
    backtracks: int
    passes: int
    grad_passes: int
    launches: int
    polish_iterations: int
    objective: float
    initial_objective: float
    kkt: float
    rel_change: float
    lambda0: float
    ms: float
    fwd_ms: float
    bwd_ms: float
    fwd_launches: int
    bwd_launches: int
    bytes: int

    @classmethod
    def from_c(cls, r: L.imrt_result) -> "Result":
        return cls(**{f.name: getattr(r, f.name) for f in dataclasses.fields(cls)})


def _ptr(a) -> int:
    """Data pointer of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr())
    return int(a.ctypes.data)


def _is_torch_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def _matrix_args(row_ptr, col, val, mask, thresholds, weights, m, n):
    """(imrt_csr, mask, thresholds, weights, arrays to keep alive) for plan_create / plan_update."""
    on_device = _is_torch_cuda(val)
    if not on_device:
        row_ptr = np.ascontiguousarray(row_ptr, np.int64)
        col = np.ascontiguousarray(col, np.int32)
        val = np.ascontiguousarray(val, np.float32)
    if not _is_torch_cuda(mask):
        mask = np.ascontiguousarray(mask, np.uint8)
    thr = np.ascontiguousarray(thresholds, np.float32)
    w = np.ascontiguousarray(weights, np.float32)
    m = int(m if m is not None else row_ptr.shape[0] - 1)
    if n is None:
        raise ValueError("n (number of beamlets) is required")
    csr = L.imrt_csr(m, int(n), int(col.shape[0]), _ptr(row_ptr), _ptr(col), _ptr(val), 1 if on_device else 0)
    return csr, mask, thr, w, (row_ptr, col, val)


class Plan:
    """One planning problem resident on the GPU (plan_create / plan_destroy)."""

    def __init__(self, row_ptr, col, val, mask, thresholds, weights, m: Optional[int] = None,
                 n: Optional[int] = None, options: Optional[Options] = None):
        lib = L.load()
        self._lib = lib
        self.options = options or Options()
        csr, mask, thr, w, keep = _matrix_args(row_ptr, col, val, mask, thresholds, weights, m, n)
        handle = ctypes.c_void_p()
        opts = self.options.to_c()
        L.check(lib.plan_create(ctypes.byref(csr), _ptr(mask), thr.shape[0], _ptr(thr), _ptr(w),
                                ctypes.byref(opts), ctypes.byref(handle)))
        self._h = handle
        self.m, self.n = csr.m, csr.n

    def update(self, row_ptr, col, val, mask, thresholds, weights, m: Optional[int] = None,
               n: Optional[int] = None) -> None:
        """plan_update: rebuilds this plan in place from a new D (sizes may change)."""
        csr, mask, thr, w, keep = _matrix_args(row_ptr, col, val, mask, thresholds, weights, m, n)
        L.check(self._lib.plan_update(self._h, ctypes.byref(csr), _ptr(mask), thr.shape[0], _ptr(thr), _ptr(w)))
        self.m, self.n = csr.m, csr.n

    def update_from_case(self, case) -> None:
        self.update(case.row_ptr, case.col, case.val, case.mask, case.thresholds, case.weights, m=case.m, n=case.n)
        vt = getattr(case, "voxel_targets", None)
        if vt is not None:
            self.set_voxel_targets(vt.dose, vt.target, vt.w_under, vt.w_over, vt.normalise)

    @classmethod
    def from_case(cls, case, options: Optional[Options] = None, device: bool = False) -> "Plan":
        """From a phantom.Case (with its voxel targets, if any); with device=True the inputs go
        through torch CUDA tensors."""
        if device:
            import torch
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            plan = cls(t(case.row_ptr), t(case.col), t(case.val), t(case.mask), case.thresholds, case.weights,
                       m=case.m, n=case.n, options=options)
        else:
            plan = cls(case.row_ptr, case.col, case.val, case.mask, case.thresholds, case.weights, m=case.m,
                       n=case.n, options=options)
        vt = getattr(case, "voxel_targets", None)
        if vt is not None:
            plan.set_voxel_targets(vt.dose, vt.target, vt.w_under, vt.w_over, vt.normalise)
        return plan

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls -------------------------------------------------------------
    def set_options(self, **changes) -> None:
        self.options = dataclasses.replace(self.options, **changes)
        opts = self.options.to_c()
        L.check(self._lib.plan_set_options(self._h, ctypes.byref(opts)))

    def set_voxel_targets(self, dose=None, target=None, w_under: float = 1.0, w_over: float = 1.0,
                          normalise: bool = False) -> None:
        """plan_set_voxel_targets: Eq. (1)'s per-voxel terms around `dose` (None removes them)."""
        if dose is not None and not _is_torch_cuda(dose):
            dose = np.ascontiguousarray(dose, np.float32)
        if target is not None and not _is_torch_cuda(target):
            target = np.ascontiguousarray(target, np.uint8)
        L.check(self._lib.plan_set_voxel_targets(self._h, _ptr(dose), _ptr(target), float(w_under), float(w_over),
                                                  1 if normalise else 0))

    def solve(self, x0=None, raise_on_error: bool = True) -> Result:
        """plan_solve; x0 (host array or CUDA tensor) is read when x_init = 2."""
        if x0 is not None and not _is_torch_cuda(x0):
            x0 = np.ascontiguousarray(x0, np.float32)
        if x0 is not None and int(x0.shape[0]) != self.n:
            raise ValueError(f"x0 has {x0.shape[0]} entries, the plan has {self.n} beamlets")
        res = L.imrt_result()
        st = self._lib.plan_solve(self._h, _ptr(x0), ctypes.byref(res))
        if raise_on_error and st not in (L.IMRT_OK,):
            L.check(st)
        return Result.from_c(res)

    def dose(self, x=None, out=None):
        """z = D x (m floats) into `out` (numpy or CUDA tensor) or a new numpy array."""
        if x is not None and not _is_torch_cuda(x):
            x = np.ascontiguousarray(x, np.float32)
        if out is None:
            out = np.empty(self.m, np.float32)
        L.check(self._lib.plan_dose(self._h, _ptr(x), _ptr(out)))
        return out

    def eval(self, x=None, z_out=None, g_out=None):
        """(G, z, g) at x: FP64 objective, dose and gradient."""
        if x is not None and not _is_torch_cuda(x):
            x = np.ascontiguousarray(x, np.float32)
        z_out = np.empty(self.m, np.float32) if z_out is None else z_out
        g_out = np.empty(self.n, np.float32) if g_out is None else g_out
        G = ctypes.c_double()
        L.check(self._lib.plan_eval(self._h, _ptr(x), ctypes.addressof(G), _ptr(z_out), _ptr(g_out)))
        return G.value, z_out, g_out

    def get_x(self, out=None):
        out = np.empty(self.n, np.float32) if out is None else out
        L.check(self._lib.plan_get_x(self._h, _ptr(out)))
        return out

    def trace(self, iterations: int, with_x: bool = False):
        """(G[k+1], lambda[k], backtracks[k], xs[k+1, n] or None) of the last solve."""
        G = np.empty(iterations + 1, np.float64)
        lam = np.empty(max(iterations, 1), np.float64)
        bt = np.empty(max(iterations, 1), np.int32)
        xs = np.empty((iterations + 1, self.n), np.float32) if with_x else None
        L.check(self._lib.plan_get_trace(self._h, iterations, _ptr(G), _ptr(lam), _ptr(bt), _ptr(xs)))
        return G, lam[:iterations], bt[:iterations], xs

    def info(self) -> dict:
        i = L.imrt_plan_info()
        L.check(self._lib.plan_info(self._h, ctypes.byref(i)))
        return {f[0]: getattr(i, f[0]) for f in L.imrt_plan_info._fields_}

    def cancel(self) -> None:
        L.check(self._lib.plan_cancel(self._h))


def version() -> str:
    return L.load().imrt_version().decode()


def trim_memory(keep_bytes: int = 0) -> None:
    """Hands the device memory the library keeps cached for later plans (current device) back
    to the system, down to `keep_bytes`."""
    L.check(L.load().imrt_trim_memory(int(keep_bytes)))


def solve_batch(plans, x0s=None, stream: int = 0, raise_on_error: bool = True):
    """plan_solve_batch: all plans in one CUDA-graph launch (one branch per plan)."""
    lib = L.load()
    n = len(plans)
    handles = (ctypes.c_void_p * n)(*[p._h.value for p in plans])
    keep = []
    x0p = None
    if x0s is not None:
        ptrs = []
        for x in x0s:
            if x is not None and not _is_torch_cuda(x):
                x = np.ascontiguousarray(x, np.float32)
            keep.append(x)
            ptrs.append(_ptr(x))
        x0p = (ctypes.c_void_p * n)(*ptrs)
    res = (L.imrt_result * n)()
    st = lib.plan_solve_batch(handles, n, x0p, res, stream)
    if raise_on_error and st != L.IMRT_OK:
        L.check(st)
    return [Result.from_c(r) for r in res]
