"""GB300-native LEEA hot path (Prellberg & Kramer, arXiv 1806.09819).

``leea`` is the ctypes binding of the CUDA library's C ABI; ``synthetic``
makes the seeded MNIST-shaped inputs; ``build`` compiles the library.  The
library is loaded lazily, on the first call that needs it.
"""
