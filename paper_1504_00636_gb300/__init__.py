"""GB300-native Voronoi particle merging (Luu, Tueckmantel & Pukhov,
arXiv:1504.00636, Sec. 3): per-cell recursive phase-space partition and
centroid merge as hand-written sm_103a CUDA kernels behind a C ABI
(``include/pma.h``).

``binding`` holds the ctypes binding (``pma_create``, ``pma_merge``, ...,
and the ``Merger`` convenience class); ``synth`` the seeded synthetic inputs.
The CUDA library is loaded on first use of the binding.
"""
from . import synth  # noqa: F401
