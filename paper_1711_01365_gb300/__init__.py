"""GB300 (sm_103a) generalized MBO diffusion-generated motion for orthogonal
matrix-valued fields on flat tori (Osting & Wang, arXiv:1711.01365).

Submodules:
  mbo     ctypes binding of the C ABI (include/mbo.h); needs the built CUDA library
  build   nvcc build of the library
  inputs  seeded synthetic initial fields
Importing the package loads nothing; ``paper_1711_01365_gb300.mbo`` loads the
CUDA library on first use and raises if it is missing.
"""
