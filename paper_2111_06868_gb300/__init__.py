"""GB300-native state-vector simulation hot path (HybridQ, arXiv 2111.06868).

The compute path is a C-ABI shared library (``libhq.so``, hand-written CUDA for
sm_103a, declared in ``include/hq.h``).  ``paper_2111_06868_gb300.hq`` is the
thin ctypes binding with the same names; ``circuits`` holds the seeded synthetic
inputs.  Importing the package does not load the CUDA library.
"""
__all__ = ["circuits", "hq"]
