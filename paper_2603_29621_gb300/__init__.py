"""GB300-native matrix-free Stokes / stabilised Navier--Stokes multigrid (libmfns).

The compute path is the CUDA library ``libmfns.so`` (C ABI in include/mfns.h);
this package holds its build script, the ctypes binding and thin Python
helpers around it.
"""
from . import _lib  # noqa: F401
