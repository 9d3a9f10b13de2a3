"""GB300-native R-matrix outer-region energy sweep.

The compute path lives in the CUDA library built from ``csrc/`` and is
reached through the ctypes binding in :mod:`paper_1403_5524_gb300.rm`.
Importing this package does not load the library; ``rm`` does, and it
raises if the library is missing (there is no CPU fallback).
"""

__all__ = ["synth", "rm"]
