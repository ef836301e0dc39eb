"""GB300-native tanTRG hot path (arXiv 2212.11973): 1-site TDVP sweeps of the
2D Hubbard half-density operator on U(1)xU(1) block-sparse MPOs.

The CUDA library (libtantrg.so, C ABI in include/tantrg.h) does all the work;
``tantrg`` is its ctypes binding, ``workloads`` the seeded input recipes.
Nothing is loaded at import time.
"""
__all__ = ["tantrg", "workloads", "build"]
