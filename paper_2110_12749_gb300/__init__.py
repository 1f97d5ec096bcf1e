"""GB300-native GSP hot path: brute-force dedispersion + single-pulse search.

The compute path is the C-ABI CUDA library libgsp.so (include/gsp.h); the
Python module ``gsp`` is a thin ctypes binding with the same entry-point
names.  Importing the package loads nothing; ``gsp.lib()`` loads the library
and raises if it has not been built.
"""
__all__ = ["gsp", "synth"]
