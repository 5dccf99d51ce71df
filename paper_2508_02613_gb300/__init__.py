"""GB300-native J-FFT solver: Green / Green-Jacobi preconditioned CG for the periodic
linear-elastic cell problem (Ladecky et al., arXiv 2508.02613), hand-written CUDA
for sm_103a behind the C ABI of include/jfft.h.

The compute path is the CUDA library ``_build/libjfft.so`` (built by ``build.build()``);
``jfft`` is its ctypes binding. Importing this package does not load the library.
"""

__all__ = ["build", "jfft"]
