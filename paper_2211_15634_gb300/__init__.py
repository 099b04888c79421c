"""GB300-native 3-D heat diffusion stencil (arXiv 2211.15634, Fig. 1).

The compute path lives in the CUDA library ``csrc/`` builds
(``libpsdiff.so``); this package only marshals arguments to its C ABI.
Submodules:

* ``inputs`` - seeded synthetic fields (no solver arithmetic).
* ``_lib``   - ctypes binding of the C ABI (loaded on first use; raises if
  the library is missing - there is no CPU fallback).
"""
__all__ = ["inputs"]
