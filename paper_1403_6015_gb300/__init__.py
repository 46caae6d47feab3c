"""GB300-native HODLR factorization of Gaussian-process covariance matrices.

The computation runs in libhodlr_gb300.so (CUDA for sm_103a) behind the C ABI declared in
include/hodlr.h; `hodlr` is its Python binding and `inputs` draws seeded synthetic inputs.
Importing this package does not load the library; `hodlr.load()` does.
"""
