"""GB300 (sm_103a) thin-film D2Q9 lattice Boltzmann library.

Implements the per-time-step hot path of Zitz et al., "A lattice Boltzmann
method for thin liquid film hydrodynamics" (arXiv:1810.07642, Section II) as
hand-written CUDA behind the C ABI of include/tflbm.h.  Submodules:
  build   compile libtflbm in-tree with nvcc (sm_103a)
  _lib    ctypes binding of the C ABI (same names as the C entry points)
  film    ThinFilm: torch-facing wrapper (device memory and streams only)
  inputs  seeded synthetic workloads shaped like the paper's simulations
The library is loaded on first use; without it every entry point raises.
"""
__all__ = ["build", "inputs"]
