"""Mixed-precision tiled Cholesky log-likelihood on NVIDIA GB300 (sm_103a).

The computation lives in libmpchol.so (C ABI: include/mpchol.h); the module
`mpchol` is its ctypes binding.  Importing this package loads nothing.
"""
