"""GB300-native parametric GEMM kernel family (arXiv 1801.04348).

`pgk` is the ctypes binding of the C ABI declared in include/pgk.h; `build`
compiles the in-tree CUDA library; `inputs` draws the seeded synthetic inputs.
Importing the package loads nothing; `pgk.lib()` loads the library and fails
loudly when it has not been built.
"""
