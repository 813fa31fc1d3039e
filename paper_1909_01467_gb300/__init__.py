"""GB300-native L-sweeps preconditioned Helmholtz solver.

The compute path is the CUDA library liblsweep.so (C ABI in include/lsweep.h); this
package holds its sources (csrc/), the in-tree build script (build.py) and the ctypes
binding (lsweep.py).  Importing the package does not load the library; the first call
through `lsweep` does, and fails loudly if it has not been built.
"""
__all__ = ["build", "lsweep"]
