"""GB300-native semiring and Strassen-Winograd matrix multiplication.

The compute path is the C-ABI shared library ``libmmsr.so`` built from
``csrc/`` (hand-written sm_103a CUDA).  ``mmsr`` is the thin ctypes binding
with the same entry-point names as ``include/mmsr.h``; ``inputs`` holds the
seeded synthetic workloads.  Importing this package loads nothing: the
library is opened on first use and raises if it has not been built.
"""
__all__ = ["mmsr", "inputs", "build"]
