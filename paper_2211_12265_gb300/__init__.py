"""Batched CRYSTALS-Dilithium (round 3) KeyGen / Sign / Verify on one GB300.

The compute path is the C-ABI library ``libdil.so`` built from ``csrc/``
(hand-written CUDA for sm_103a).  ``paper_2211_12265_gb300.dil`` is the thin
ctypes binding with the same names as the C entry points; ``workload`` holds the
seeded synthetic-input generators.  Importing this package loads nothing: the
binding loads the library on first use and raises if it is missing.
"""

__all__ = ["dil", "workload", "serving"]
