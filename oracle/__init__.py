"""FP64 CPU oracle of the IMRT fluence-map optimiser (Men et al., arXiv:0908.4421).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg, never by the library. It shares no code
with the CUDA path; both sides receive the same arrays from the input generator.

The arithmetic lives in ``oracle.c`` (plain loops in double precision; see its
header for the equations and readings it follows). This module only marshals
numpy arrays into it.

Parity status: every function here is pinned by tests that do not re-use the
oracle's own formulas (finite differences, brute-force NNLS, an independent
bound-constrained solver, closed forms, dense library products, invariants).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, ENOMEM, ELINESEARCH = 0, 1, 2, 4
STOP_REL, STOP_MAXITER, STOP_EXACT, STOP_STATIONARY = 1, 2, 3, 4


def build(force: bool = False, src: str = _SRC, out: str = _LIB, extra_flags=()) -> str:
    """Compiles oracle.c (gcc -O2, OpenMP, no FP contraction) into a shared library."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
                               *extra_flags, "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


class _Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("n_structures", ctypes.c_int32),
                ("thresholds", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("vt", ctypes.c_void_p), ("vt_target", ctypes.c_void_p),
                ("vt_wu", ctypes.c_double), ("vt_wo", ctypes.c_double), ("vt_normalise", ctypes.c_int32)]


class _Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("alpha", ctypes.c_double), ("lambda0", ctypes.c_double),
                ("delta", ctypes.c_double), ("max_iter", ctypes.c_int32), ("max_backtracks", ctypes.c_int32),
                ("x_init", ctypes.c_int32), ("threads", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("backtracks", ctypes.c_int32),
                ("stop_reason", ctypes.c_int32), ("objective", ctypes.c_double), ("kkt", ctypes.c_double),
                ("rel_change", ctypes.c_double), ("lambda0", ctypes.c_double),
                ("initial_objective", ctypes.c_double)]


class _Trace(ctypes.Structure):
    _fields_ = [("G", ctypes.c_void_p), ("lam", ctypes.c_void_p), ("backtracks", ctypes.c_void_p),
                ("x", ctypes.c_void_p)]


class Oracle:
    """ctypes handle to one compiled oracle library (the default, or a test build)."""

    def __init__(self, path: Optional[str] = None):
        lib = ctypes.CDLL(path or build())
        P = ctypes.POINTER
        lib.orc_solve.restype = ctypes.c_int
        lib.orc_solve.argtypes = [P(_Problem), P(_Params), ctypes.c_void_p, P(_Trace), P(_Result)]
        lib.orc_eval.restype = ctypes.c_double
        lib.orc_eval.argtypes = [P(_Problem), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_int32]
        lib.orc_lambda0.restype = ctypes.c_double
        lib.orc_lambda0.argtypes = [P(_Problem), ctypes.c_int32, ctypes.c_int32]
        lib.orc_initial_point.restype = None
        lib.orc_initial_point.argtypes = [P(_Problem), ctypes.c_int32, ctypes.c_void_p]
        self._lib = lib

    @staticmethod
    def _problem(case):
        keep = dict(row_ptr=np.ascontiguousarray(case.row_ptr, np.int64),
                    col=np.ascontiguousarray(case.col, np.int32),
                    val=np.ascontiguousarray(case.val, np.float32),
                    mask=np.ascontiguousarray(case.mask, np.uint8),
                    thr=np.ascontiguousarray(case.thresholds, np.float32),
                    w=np.ascontiguousarray(case.weights, np.float32))
        vt = getattr(case, "voxel_targets", None)
        vt_ptr = vt_tg = None
        wu = wo = 0.0
        norm = 0
        if vt is not None:
            keep["vt"] = np.ascontiguousarray(vt.dose, np.float32)
            keep["vtg"] = np.ascontiguousarray(vt.target, np.uint8)
            vt_ptr, vt_tg = keep["vt"].ctypes.data, keep["vtg"].ctypes.data
            wu, wo, norm = float(vt.w_under), float(vt.w_over), int(vt.normalise)
        p = _Problem(case.m, case.n, keep["row_ptr"].ctypes.data, keep["col"].ctypes.data,
                     keep["val"].ctypes.data, keep["mask"].ctypes.data, case.n_structures,
                     keep["thr"].ctypes.data, keep["w"].ctypes.data, vt_ptr, vt_tg, wu, wo, norm)
        return p, keep

    def eval(self, case, x, gradient: bool = True, threads: int = 0):
        """(G, z, r, g) at x in FP64 (Eq. (1)-(4))."""
        p, keep = self._problem(case)
        x = np.ascontiguousarray(x, np.float64)
        z = np.empty(case.m, np.float64)
        r = np.empty(case.m, np.float64)
        g = np.empty(case.n, np.float64) if gradient else None
        G = self._lib.orc_eval(ctypes.byref(p), x.ctypes.data, z.ctypes.data, r.ctypes.data,
                               g.ctypes.data if gradient else None, threads)
        return G, z, r, g

    def dose(self, case, x, threads: int = 0):
        return self.eval(case, x, gradient=False, threads=threads)[1]

    def lambda0_rule(self, case, iters: int = 50, threads: int = 0) -> float:
        p, keep = self._problem(case)
        return float(self._lib.orc_lambda0(ctypes.byref(p), iters, threads))

    def initial_point(self, case, x_init: int = 0):
        p, keep = self._problem(case)
        x = np.empty(case.n, np.float64)
        self._lib.orc_initial_point(ctypes.byref(p), x_init, x.ctypes.data)
        return x

    def solve(self, case, lambda0: float = 0.0, eps: float = 1e-4, alpha: float = 2.0, delta: float = 1e-6,
              max_iter: int = 200, max_backtracks: int = 50, x_init: int = 0, x0=None, threads: int = 0,
              trace: bool = True, trace_x: bool = False) -> "SolveResult":
        """Runs the projected-gradient Armijo loop (Sec. 2.2) and returns the trajectory."""
        p, keep = self._problem(case)
        q = _Params(eps, alpha, lambda0, delta, max_iter, max_backtracks, x_init, threads)
        x = np.zeros(case.n, np.float64) if x0 is None else np.array(x0, np.float64)
        tG = np.full(max_iter + 1, np.nan) if trace else None
        tl = np.full(max_iter, np.nan) if trace else None
        tb = np.full(max_iter, -1, np.int32) if trace else None
        tx = np.full((max_iter + 1, case.n), np.nan) if trace_x else None
        tr = _Trace(tG.ctypes.data if trace else None, tl.ctypes.data if trace else None,
                    tb.ctypes.data if trace else None, tx.ctypes.data if trace_x else None)
        res = _Result()
        self._lib.orc_solve(ctypes.byref(p), ctypes.byref(q), x.ctypes.data, ctypes.byref(tr), ctypes.byref(res))
        k = res.iterations
        return SolveResult(status=res.status, iterations=k, backtracks=res.backtracks,
                           stop_reason=res.stop_reason, objective=res.objective, kkt=res.kkt,
                           rel_change=res.rel_change, lambda0=res.lambda0,
                           initial_objective=res.initial_objective, x=x,
                           G=tG[:k + 1] if trace else None, lambdas=tl[:k] if trace else None,
                           backtrack_trace=tb[:k] if trace else None,
                           xs=tx[:k + 1] if trace_x else None)


@dataclasses.dataclass
class SolveResult:
    status: int
    iterations: int
    backtracks: int
    stop_reason: int
    objective: float
    kkt: float
    rel_change: float
    lambda0: float
    initial_objective: float
    x: np.ndarray
    G: Optional[np.ndarray]
    lambdas: Optional[np.ndarray]
    backtrack_trace: Optional[np.ndarray]
    xs: Optional[np.ndarray]


_default: Optional[Oracle] = None


def get() -> Oracle:
    """The oracle built from oracle.c (compiled on first use)."""
    global _default
    if _default is None:
        _default = Oracle()
    return _default
