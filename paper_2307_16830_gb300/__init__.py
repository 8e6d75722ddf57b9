"""GB300-native (sm_103a, FP64) ACOPF callbacks and condensed-KKT assembly.

The compute path lives in the CUDA/C++ shared library ``libacopf.so`` built
from ``csrc/``; ``paper_2307_16830_gb300.acopf`` is its thin ctypes binding.
Importing this package does not load the library; ``synth`` (seeded synthetic
grids and points) needs only numpy.
"""
__all__ = ["acopf", "synth"]
