"""GB300-native EAM hot path of the MOLDY method.

The compute lives in a C-ABI CUDA library (include/md.h, csrc/); `md` is its
thin ctypes binding and `inputs` builds seeded synthetic workloads.  Importing
the package loads nothing; the first call into `md` loads the library and fails
loudly if it has not been built.
"""
__all__ = ["inputs", "md"]
