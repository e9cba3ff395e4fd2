"""GB300-native hot path of the sampling-based finite-PEPS optimiser (arXiv:2503.12557).

The compute runs in hand-written sm_103a CUDA kernels behind a C ABI (``include/peps_gb300.h``);
``paper_2503_12557_gb300.peps`` is the thin ctypes binding over it.  ``inputs`` holds the seeded
synthetic-input generators.  Importing this package loads nothing compiled: the binding loads
the shared library on first use and raises if it is missing.
"""
__all__ = ["inputs", "peps"]
