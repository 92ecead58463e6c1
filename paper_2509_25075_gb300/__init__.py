"""GB300 (sm_103a) library for the GEM hot path (arXiv 2509.25075).

* ``binding``   -- ctypes binding of the C ABI in include/gem.h (``Context``,
                   ``GemLoss``); every step runs in libgem.so.
* ``synthetic`` -- seeded synthetic inputs (no method arithmetic).
* ``build``     -- in-tree nvcc build of libgem.so for sm_103a.

Importing the package does not load CUDA; the library is loaded on first use.
"""

__all__ = ["binding", "synthetic", "build"]
