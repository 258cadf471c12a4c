"""Restarted mixed-precision CG with a kNN-chosen switch tolerance, for GB300.

Method: Prolubnikov, "Parameter Optimization for Restarted Mixed-Precision
Iterative Sparse Solver" (arXiv 2412.08059).  The solver is the CUDA library
libmpcg.so (C ABI in include/mpcg.h, sources in csrc/); `mpcg` is its ctypes
binding over torch device memory and streams; `build.build()` compiles it.
"""
from . import build, mpcg  # noqa: F401
