"""GB300-native superfast Tikhonov regularisation of Toeplitz systems (arXiv 1302.6945, l2 penalty).

The solver lives in the CUDA library libtikh.so (C-ABI in include/tikh.h); ``tikh`` is its Python
binding and ``workloads`` draws seeded synthetic inputs.  Importing the package loads nothing; the
binding loads the library on first use and raises if it has not been built.
"""
