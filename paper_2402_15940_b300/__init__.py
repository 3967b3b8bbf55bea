"""B300-native matrix-free partial-assembly finite elements (arXiv 2402.15940, hot path).

The compute path is libfepa.so (hand-written sm_103a CUDA behind a C ABI, see
include/fepa.h); this package is its thin Python binding.
"""
from .fepa import (DIFFUSION, MASS, PRECOND_JACOBI, PRECOND_NONE, Batch, CgStats, FepaError, Multigrid,
                   Operator, hex_numbering, launch_count, load_library, LIB_PATH)

__all__ = ["Operator", "Batch", "Multigrid", "FepaError", "CgStats", "MASS", "DIFFUSION", "PRECOND_NONE", "PRECOND_JACOBI",
           "hex_numbering", "launch_count", "load_library", "LIB_PATH"]
