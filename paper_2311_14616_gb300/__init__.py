"""GB300-native mixed-precision iterative refinement (Kelley, arXiv 2311.14616).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/ir.h``); ``ir`` is its ctypes binding.  Importing this package does
not load the library; the first call does, and raises if it is not built.
"""
from .ir import (BF16, F16, F32, F64, TF32, Context, Factorization, IRError, Report,  # noqa: F401
                 default_term, lib)

__all__ = ["Context", "Factorization", "IRError", "Report", "default_term", "lib",
           "F64", "F32", "TF32", "BF16", "F16"]
