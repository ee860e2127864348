"""GB300-native ordinary kriging of missing inter-slice voxels (arXiv 2303.09523).

The compute path is the CUDA library ``libkrig.so`` built from ``csrc/`` and
called through its C ABI (declared in ``include/krig.h``).  ``binding`` is the
thin ctypes layer over it; ``phantoms`` generates seeded synthetic slice stacks.
Importing this package does not load the library; ``binding.lib()`` does, and
raises if it is missing.
"""
__all__ = ["binding", "phantoms"]
