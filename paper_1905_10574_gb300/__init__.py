"""GB300-native robust tiled solver for the triangular Sylvester equation
A*Y + Y*B = alpha*C (Schwarz & Kjelgaard Mikkelsen, 2019).

The compute path is the CUDA library ``_build/libsylv.so`` (C ABI declared in
``include/sylv.h``); ``sylv`` is its thin ctypes binding and ``inputs`` the seeded
workload generators.  Importing the package does not load the library; the first
call into ``sylv`` does, and raises if it has not been built.
"""
__all__ = ["inputs", "sylv"]
