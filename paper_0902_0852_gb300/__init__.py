"""GB300-native extended-precision Cholesky and inverse iteration for the
Hankel moment matrices of Emmart, Weems and Chen.

The compute path is the CUDA library ``libhk.so`` behind the C ABI in
``include/hk.h``; ``hk`` is its Python binding and ``inputs`` the seeded input
generator (moments).  Importing the package loads nothing heavy.
"""
__all__ = ["hk", "inputs", "build"]
