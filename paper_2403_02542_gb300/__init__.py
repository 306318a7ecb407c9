"""GB300-native walker step of large-time-step phaseless AFQMC.

The computation lives in the CUDA library libafqmc.so (C ABI in
include/afqmc.h); this package holds its ctypes binding (``api``), the build
script (``build``) and the seeded synthetic inputs (``inputs``).  Importing
the package does not load the library; ``api.Context`` does, and fails loudly
when it has not been built.
"""
__all__ = ["api", "build", "inputs"]
