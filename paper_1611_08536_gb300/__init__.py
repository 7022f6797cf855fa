"""GB300-native DRTS time step (arXiv:1611.08536): x_{t+1} = A x_t + s(t).

The compute path is the CUDA library ``libdrts.so`` (sources in ``csrc/``,
C ABI in ``include/drts.h``); ``drts`` is its thin ctypes binding.  Importing
this package does not load the library; ``paper_1611_08536_gb300.drts`` does,
and fails loudly when it is missing.
"""
__all__ = ["inputs", "drts"]
