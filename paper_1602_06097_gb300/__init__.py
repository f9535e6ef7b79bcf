"""GB300-native Faugere-Lachartre reduction over GF(p), p < 2^16.

The reduction runs in hand-written CUDA kernels for sm_103a behind the C ABI
declared in ``include/gbla.h``; :mod:`paper_1602_06097_gb300.gbla` is the thin
ctypes binding over it and :mod:`paper_1602_06097_gb300.synth` draws seeded
synthetic F4-shaped inputs.  Importing the package loads nothing native: the
shared library is opened on first use of the binding.
"""
__all__ = ["gbla", "synth"]
