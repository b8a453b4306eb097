"""GB300-native supernodal sparse Cholesky (arXiv 1608.00044, fan-both method).

The compute path is the native library ``libspchol.so`` (CUDA for sm_103a plus
host C++ symbolic analysis) behind the C-ABI of ``include/spchol.h``;
``spchol`` is its ctypes binding.
"""
from . import spchol
from .spchol import (
    FP32,
    FP64,
    TF32,
    TF32X3,
    FP64_TC,
    SparseCholesky,
    SpcholError,
    analyze,
    batch_analyze,
    batch_factorize,
    batch_info,
    batch_solve,
    default_options,
    destroy,
    export_factor,
    factorize,
    solve,
    stats,
    strerror,
)

__all__ = [
    "spchol",
    "FP32",
    "FP64",
    "TF32",
    "TF32X3",
    "FP64_TC",
    "SparseCholesky",
    "SpcholError",
    "analyze",
    "batch_analyze",
    "batch_factorize",
    "batch_info",
    "batch_solve",
    "default_options",
    "destroy",
    "export_factor",
    "factorize",
    "solve",
    "stats",
    "strerror",
]
