"""GB300 (sm_103a) Spectral Difference Raviart-Thomas residual library.

The compute path is libsdrt.so (CUDA C++, C ABI in include/sdrt.h); `sdrt`
is its ctypes binding.  Build the library with `build.build()`.
"""
