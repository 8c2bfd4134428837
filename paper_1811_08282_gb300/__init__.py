"""GB300-native swept time-space decomposition for explicit 1D stencils.

The compute path lives in the CUDA library ``libswept.so`` (``csrc/``) behind a
C ABI declared in ``include/swept.h``; ``swept`` is its thin ctypes binding.
``inputs`` holds the seeded synthetic problem generators.
"""
