"""GB300-native collective multigrid for PDE-constrained optimisation under
uncertainty (linear-quadratic elliptic control, arXiv 2302.13680).

The compute path is libcmg.so (CUDA, sm_103a) behind the C ABI in
include/cmg.h; this package holds its sources, its build and a thin ctypes
binding.
"""
from .cmg import (Batch, BoundaryHierarchy, CMGError, CycleOptions, Hierarchy, load_library, LIB_PATH, FP32, FP64,  # noqa: F401
                  METHOD_CYCLE, METHOD_FGMRES, SMOOTH_JACOBI, SMOOTH_RBGS, BATCH_AUTO, BATCH_PERSISTENT,
                  BATCH_BRANCHES, BATCH_LEGS_BY_WORK, BATCH_LEGS_PERSISTENT, BATCH_LEGS_PHASES)
