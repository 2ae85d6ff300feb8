"""GB300 (sm_103a) implementation of the WCSPH time step with the generalised
wall boundary treatment of Rezavand, Zhang & Hu (arXiv 2110.02621).

The method runs in the CUDA library ``_build/libsph_gb300.so`` behind the C ABI
of ``include/sph.h``; ``sph`` is its ctypes binding, ``scenes`` generates the
seeded synthetic particle inputs, ``build`` compiles the library.
"""
from . import scenes  # noqa: F401

__all__ = ["scenes", "sph", "build"]
