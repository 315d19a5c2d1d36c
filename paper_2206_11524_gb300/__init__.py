"""GB300 (sm_103a) homogenized multi-component Shan-Chen lattice Boltzmann
library (HMCSC, arXiv 2206.11524).

Submodules:
  lbm     ctypes binding of the C ABI in include/lbm.h (+ ``Lattice`` wrapper)
  build   nvcc build of the CUDA library
  synth   seeded synthetic inputs (geometry, wettability, densities)
  params  host-side parameter conversions (contact angle, viscosity)
  serve   continuous-batching server of independent simulations
  autotune  launch-shape autotuner with a persisted table
"""
__all__ = ["lbm", "build", "synth", "params", "serve", "autotune"]
