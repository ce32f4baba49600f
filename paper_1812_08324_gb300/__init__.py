"""GB300-native H-matrix Crank-Nicolson solver for Levy-process generators.

The compute path is the CUDA library ``_build/liblevyhm.so`` (C ABI declared in
``include/levy_hmat.h``); ``hmat`` is a thin ctypes binding over it.  Importing
this package does not load the library; ``hmat.load()`` does, and raises if
the library is missing -- there is no CPU fallback.
"""
__all__ = ["hmat", "workloads", "build"]
