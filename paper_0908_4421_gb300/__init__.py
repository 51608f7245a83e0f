"""GB300-native penalty-based quadratic fluence-map optimiser.

Men et al., "GPU-based ultra fast IMRT plan optimization" (arXiv:0908.4421):
gradient projection with Armijo's line search on beamlet intensities x >= 0,
with the sparse dose product z = D x and the gradient D^T r as hand-written
sm_103a CUDA kernels behind a C ABI (include/imrt.h, libimrt.so).

Importing the package does not load the CUDA library; creating a Plan does,
and fails loudly if libimrt.so has not been built.
"""
from .api import Options, Plan, Result, solve_batch, trim_memory, version  # noqa: F401
from . import _lib  # noqa: F401
