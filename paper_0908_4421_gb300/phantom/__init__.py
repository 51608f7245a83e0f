"""Seeded synthetic prostate phantom and dose-deposition matrix (input generator).

The paper's test case (Sec. 3.1, Table 1) is a clinical prostate plan that is
not available; these phantoms stand in for it with matching shapes: nine (or
five) coplanar beams, a PTV abutted by the rectum, the bladder
anterior-superior, and a body contour, on 5 mm / 2.5 mm voxel grids.

This module generates INPUTS only: the voxel-major CSR matrix D (Sec. 2.1:
z_j = sum_i D_ij x_i), the structure bitmask, and the raw per-structure dose
thresholds and weights. It holds none of the optimiser's arithmetic (no
penalties, no normalisation, no gradient); the CUDA library and the FP64
oracle each do that themselves. Random draws (configs with jitter) come from
numpy's PCG64 seeded per case.

The heavy lifting is in ``phantom.c`` (OpenMP, -ffp-contract=off), compiled on
first use or by ``__graft_entry__.build()``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from typing import Dict, List, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phantom.c")
_LIB = os.path.join(_HERE, "libphantom.so")

# Structure bits of the per-voxel mask (bit s set => voxel in structure s).
STRUCTURES = ("PTV", "rectum", "bladder", "body")
NAN = float("nan")


@dataclasses.dataclass(frozen=True)
class PhantomSpec:
    """Geometry and dose-kernel parameters of one synthetic case (mm, Gy)."""

    shape: Tuple[int, int, int] = (40, 40, 30)
    spacing: float = 5.0
    body_axes: Tuple[float, float] = (90.0, 70.0)
    ptv_radii: Tuple[float, float, float] = (25.0, 20.0, 20.0)
    ptv_centre: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    rectum_radius: float = 10.0
    rectum_y: float = -30.0
    rectum_z: Tuple[float, float] = (-40.0, 40.0)
    bladder_radius: float = 22.0
    bladder_centre: Tuple[float, float, float] = (0.0, 20.0, 30.0)
    n_beams: int = 5
    angle0_deg: float = 0.0
    beamlet_mm: float = 5.0
    margin_mm: float = 5.0
    mu_per_mm: float = 0.005
    sigma_mm: float = 2.5
    cutoff: float = 1e-3
    coarse_unspecified: bool = False  # unspecified tissue only on the 2x coarser grid (Sec. 3.1)
    # per-structure (under, over) thresholds in Gy (NaN: no term) and weights
    thresholds: Tuple[Tuple[float, float], ...] = ((76.0, 78.0), (NAN, 40.0), (NAN, 45.0), (NAN, 30.0))
    weights: Tuple[Tuple[float, float], ...] = ((100.0, 100.0), (0.0, 10.0), (0.0, 5.0), (0.0, 1.0))


class _CSpec(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("spacing", ctypes.c_double),
        ("body_a", ctypes.c_double), ("body_b", ctypes.c_double),
        ("ptv_r", ctypes.c_double * 3), ("ptv_c", ctypes.c_double * 3),
        ("rect_r", ctypes.c_double), ("rect_y", ctypes.c_double),
        ("rect_z0", ctypes.c_double), ("rect_z1", ctypes.c_double),
        ("blad_r", ctypes.c_double), ("blad_c", ctypes.c_double * 3),
        ("n_beams", ctypes.c_int32),
        ("angle0_deg", ctypes.c_double), ("beamlet_mm", ctypes.c_double),
        ("margin_mm", ctypes.c_double), ("mu_per_mm", ctypes.c_double),
        ("sigma_mm", ctypes.c_double), ("cutoff", ctypes.c_double),
        ("coarse_unspecified", ctypes.c_int32),
    ]


def _to_c(s: PhantomSpec) -> _CSpec:
    c = _CSpec()
    c.nx, c.ny, c.nz = s.shape
    c.spacing = s.spacing
    c.body_a, c.body_b = s.body_axes
    c.ptv_r = (ctypes.c_double * 3)(*s.ptv_radii)
    c.ptv_c = (ctypes.c_double * 3)(*s.ptv_centre)
    c.rect_r, c.rect_y = s.rectum_radius, s.rectum_y
    c.rect_z0, c.rect_z1 = s.rectum_z
    c.blad_r = s.bladder_radius
    c.blad_c = (ctypes.c_double * 3)(*s.bladder_centre)
    c.n_beams = s.n_beams
    c.angle0_deg = s.angle0_deg
    c.beamlet_mm = s.beamlet_mm
    c.margin_mm = s.margin_mm
    c.mu_per_mm = s.mu_per_mm
    c.sigma_mm = s.sigma_mm
    c.cutoff = s.cutoff
    c.coarse_unspecified = 1 if s.coarse_unspecified else 0
    return c


def build_native(force: bool = False) -> str:
    """Compiles phantom.c into libphantom.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib_handle: Optional[ctypes.CDLL] = None


def _lib() -> ctypes.CDLL:
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build_native())
        P = ctypes.POINTER
        lib.phantom_count_body.restype = ctypes.c_int64
        lib.phantom_count_body.argtypes = [P(_CSpec)]
        lib.phantom_fill_voxels.restype = None
        lib.phantom_fill_voxels.argtypes = [P(_CSpec), ctypes.c_void_p, ctypes.c_void_p]
        lib.phantom_count_beamlets.restype = ctypes.c_int32
        lib.phantom_count_beamlets.argtypes = [P(_CSpec)]
        lib.phantom_fill_beamlets.restype = None
        lib.phantom_fill_beamlets.argtypes = [P(_CSpec), ctypes.c_void_p]
        lib.phantom_count_rows.restype = None
        lib.phantom_count_rows.argtypes = [P(_CSpec), ctypes.c_int64, ctypes.c_void_p]
        lib.phantom_fill_rows.restype = None
        lib.phantom_fill_rows.argtypes = [P(_CSpec), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]
        _lib_handle = lib
    return _lib_handle


@dataclasses.dataclass
class VoxelTargets:
    """Per-voxel dose targets of Eq. (1) as printed: T_j is the original plan's dose, V_T the
    target voxels (under-dose term), every voxel carries the over-dose term."""

    dose: np.ndarray        # float32 [m], T_j
    target: np.ndarray      # uint8 [m], 1 => j in V_T
    w_under: float = 1.0
    w_over: float = 1.0
    normalise: bool = False  # divide the terms by |V_T| and m


@dataclasses.dataclass
class Case:
    """One generated planning problem (host arrays)."""

    spec: PhantomSpec
    row_ptr: np.ndarray      # int64 [m+1]
    col: np.ndarray          # int32 [nnz]
    val: np.ndarray          # float32 [nnz]
    mask: np.ndarray         # uint8 [m], bit s => structure s
    thresholds: np.ndarray   # float32 [S, 2] (under, over); NaN => no term
    weights: np.ndarray      # float32 [S, 2]
    voxels: np.ndarray       # float32 [m, 3] voxel centres (mm)
    beamlets: np.ndarray     # float32 [n, 3] (beam, u, v)
    voxel_targets: Optional[VoxelTargets] = None

    @property
    def m(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def n(self) -> int:
        return int(self.beamlets.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def n_structures(self) -> int:
        return int(self.thresholds.shape[0])


def make_case(spec: PhantomSpec) -> Case:
    """Generates D (voxel-major CSR, FP32 values, int32 columns) and the structures."""
    lib = _lib()
    cs = _to_c(spec)
    m = int(lib.phantom_count_body(ctypes.byref(cs)))
    voxels = np.empty((m, 3), np.float32)
    mask = np.empty(m, np.uint8)
    lib.phantom_fill_voxels(ctypes.byref(cs), voxels.ctypes.data, mask.ctypes.data)
    n = int(lib.phantom_count_beamlets(ctypes.byref(cs)))
    beamlets = np.empty((n, 3), np.float32)
    lib.phantom_fill_beamlets(ctypes.byref(cs), beamlets.ctypes.data)
    counts = np.empty(m, np.int64)
    lib.phantom_count_rows(ctypes.byref(cs), m, counts.ctypes.data)
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float32)
    lib.phantom_fill_rows(ctypes.byref(cs), m, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data)
    thr = np.array(spec.thresholds, np.float32).reshape(-1, 2)
    w = np.array(spec.weights, np.float32).reshape(-1, 2)
    return Case(spec, row_ptr, col, val, mask, thr, w, voxels, beamlets)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

#: 40x40x30 voxels at 5 mm, 5 coplanar beams at 0, 72, ..., 288 deg, 5x5 mm beamlets.
TINY_5MM_5BEAM = PhantomSpec()

#: 192x160x96 voxels at 2.5 mm, 9 beams at 40 deg steps, 5x5 mm beamlets,
#: the 2.5 mm lateral kernel cut at 1e-3 (about 2.5M nonzeros: L2-resident).
PROSTATE_2P5MM_9BEAM = dataclasses.replace(
    TINY_5MM_5BEAM, shape=(192, 160, 96), spacing=2.5, n_beams=9)

#: The same grid and beams with 2.5x2.5 mm beamlets, a 6 mm lateral kernel and a
#: 1e-4 cut, which puts D in the 50-150M nonzero band of the paper's largest
#: scenario (Table 1 row 3: 43M) and far above the 129 MB L2.
PROSTATE_2P5MM_9BEAM_L = dataclasses.replace(
    PROSTATE_2P5MM_9BEAM, beamlet_mm=2.5, sigma_mm=6.0, cutoff=1e-4)

#: The literal paper-shaped grid with the unspecified tissue on the 2x coarser grid (Sec. 3.1).
PROSTATE_2P5MM_9BEAM_MIXED = dataclasses.replace(PROSTATE_2P5MM_9BEAM, coarse_unspecified=True)

WORKLOADS: Dict[str, PhantomSpec] = {
    "tiny-40x40x30-5mm-5beam": TINY_5MM_5BEAM,
    "prostate-192x160x96-2.5mm-9beam": PROSTATE_2P5MM_9BEAM,
    "prostate-192x160x96-2.5mm-9beam-2.5mm-beamlets": PROSTATE_2P5MM_9BEAM_L,
    "prostate-192x160x96-2.5mm-9beam-mixed-resolution": PROSTATE_2P5MM_9BEAM_MIXED,
}


def with_voxel_targets(case: Case, dose: np.ndarray, target: Optional[np.ndarray] = None, w_under: float = 1.0,
                       w_over: float = 1.0, normalise: bool = False) -> Case:
    """A copy of `case` whose objective also carries Eq. (1)'s per-voxel terms around `dose`
    (default V_T: the PTV, structure bit 0)."""
    if target is None:
        target = (case.mask & 1).astype(np.uint8)
    vt = VoxelTargets(np.ascontiguousarray(dose, np.float32), np.ascontiguousarray(target, np.uint8),
                      float(w_under), float(w_over), bool(normalise))
    return dataclasses.replace(case, voxel_targets=vt)


def jittered_spec(seed: int, shift_mm: float = 0.0, base: PhantomSpec = TINY_5MM_5BEAM,
                  vary: bool = True) -> PhantomSpec:
    """A seeded variant of `base` for batched and streaming workloads.

    With ``vary``: voxel spacing from {2.5, 4, 5} mm (same physical extent as the
    base grid), beam count from {5, 7, 9}, beamlet pitch from {5, 10} mm, and PTV
    radii scaled uniformly in [0.8, 1.2]. ``shift_mm`` > 0 also moves the PTV by
    a uniform offset in [-shift_mm, shift_mm] per axis.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    s = base
    if vary:
        spacing = float(rng.choice([2.5, 4.0, 5.0]))
        extent = [base.shape[i] * base.spacing for i in range(3)]
        shape = tuple(int(round(e / spacing)) for e in extent)
        scale = float(rng.uniform(0.8, 1.2))
        s = dataclasses.replace(
            s, shape=shape, spacing=spacing, n_beams=int(rng.choice([5, 7, 9])),
            beamlet_mm=float(rng.choice([5.0, 10.0])),
            ptv_radii=tuple(r * scale for r in base.ptv_radii))
    if shift_mm > 0:
        off = rng.uniform(-shift_mm, shift_mm, size=3)
        s = dataclasses.replace(s, ptv_centre=tuple(float(c + o) for c, o in zip(s.ptv_centre, off)))
    return s


def csr_to_dense(case: Case) -> np.ndarray:
    """Dense FP64 copy of D (m x n) for tiny cases in tests."""
    d = np.zeros((case.m, case.n), np.float64)
    for j in range(case.m):
        a, b = case.row_ptr[j], case.row_ptr[j + 1]
        d[j, case.col[a:b]] = case.val[a:b]
    return d


def random_case(seed: int, m: int, n: int, density: float, n_structures: int = 2,
                empty_rows: int = 0, long_rows: int = 0, value_scale: float = 1.0) -> Case:
    """A random sparse problem with ragged rows for kernel and solver tests.

    ``empty_rows`` rows get no entries; ``long_rows`` rows are fully dense.
    Structure 0 carries an under- and over-dose term, the others over-dose only.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    rows: List[np.ndarray] = []
    vals: List[np.ndarray] = []
    dense_rows = set(rng.choice(m, size=min(long_rows, m), replace=False).tolist()) if long_rows else set()
    others = np.array([j for j in range(m) if j not in dense_rows], np.int64)
    empty = set(rng.choice(others, size=min(empty_rows, others.size), replace=False).tolist()) if empty_rows else set()
    for j in range(m):
        if j in empty:
            c = np.zeros(0, np.int64)
        elif j in dense_rows:
            c = np.arange(n)
        else:
            k = int(rng.binomial(n, density))
            c = np.sort(rng.choice(n, size=k, replace=False))
        rows.append(c.astype(np.int32))
        vals.append((rng.uniform(0.05, 1.0, size=c.size) * value_scale).astype(np.float32))
    counts = np.array([r.size for r in rows], np.int64)
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = np.concatenate(rows) if rows else np.zeros(0, np.int32)
    val = np.concatenate(vals) if vals else np.zeros(0, np.float32)
    mask = np.zeros(m, np.uint8)
    for s in range(n_structures):
        member = rng.uniform(size=m) < (0.35 if s == 0 else 0.5)
        mask |= (member.astype(np.uint8) << s)
    mask[mask == 0] = 1 << (n_structures - 1)
    thr = np.full((n_structures, 2), np.nan, np.float32)
    w = np.zeros((n_structures, 2), np.float32)
    thr[0] = (float(rng.uniform(0.8, 1.2)), float(rng.uniform(1.3, 1.6)))
    w[0] = (float(rng.uniform(1, 10)), float(rng.uniform(1, 10)))
    for s in range(1, n_structures):
        thr[s, 1] = float(rng.uniform(0.2, 0.8))
        w[s, 1] = float(rng.uniform(0.5, 5))
    spec = dataclasses.replace(TINY_5MM_5BEAM, thresholds=tuple(map(tuple, thr.tolist())),
                               weights=tuple(map(tuple, w.tolist())))
    voxels = np.zeros((m, 3), np.float32)
    beamlets = np.zeros((n, 3), np.float32)
    return Case(spec, row_ptr, col.astype(np.int32), val, mask, thr, w, voxels, beamlets)
