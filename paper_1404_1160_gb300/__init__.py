"""GB300-native improved-ETD particle-in-cell library (Frenod, Hirstoaga & Lutz).

The compute path is the C-ABI library ``libpic.so`` (hand-written CUDA for
sm_103a) declared in ``include/pic.h``; ``paper_1404_1160_gb300.pic`` is its
thin ctypes binding.  Importing this package loads nothing; the binding loads
the library on first use and raises if it is missing.
"""
__all__ = ["pic", "inputs"]
