"""GB300 (sm_103a) sparsify-and-solve library: GRASS similarity-aware spectral
sparsification (arXiv 1911.04382) and sparsifier-preconditioned PCG.

The compute path is libgrass.so (hand-written CUDA behind the C ABI of
include/grass.h); this package holds its sources (csrc/), the in-tree build
(build.py) and the ctypes binding (binding.py, same names as the C ABI).
"""
from .build import build, LIB  # noqa: F401
from .binding import *  # noqa: F401,F403
from .binding import lib, GrassError, make_params  # noqa: F401
