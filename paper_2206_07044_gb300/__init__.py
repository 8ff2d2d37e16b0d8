"""GB300 engine for hyper-optimized approximate tensor-network contraction.

The hot path -- executing a frozen ordered contraction tree of pairwise
contractions and QR/LQ/SVD bond compressions down to log|Z| -- runs in the
CUDA library ``libtn.so`` (C ABI in include/tn.h); ``tn`` is its ctypes
binding.  Build the library with ``paper_2206_07044_gb300.build.build()``.
"""
from .tn import Context, TNError, lib, version  # noqa: F401
