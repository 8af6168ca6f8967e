"""GB300 (sm_103a) 3D RSF level-set evolution (arXiv 2404.02813).

The compute path is librsf.so (CUDA, C ABI in include/rsf.h); this package
holds its build step (``build``), the ctypes binding (``rsf``) and the seeded
synthetic inputs (``synth``).  Importing it does not load the library; the
first call does, and fails loudly if it has not been built.
"""
from .rsf import Context, Params, RSFError, context, evolve, load_library  # noqa: F401
