"""GB300-native differentiable spherical 2D-Gaussian rasterizer (Splat-LOAM, arXiv 2503.17491).

The compute path is libsplatloam (hand-written sm_103a CUDA behind the C ABI in
include/splatloam.h).  Submodules: ``_lib`` (ctypes binding of the C ABI), ``api`` (PyTorch
layer: contexts, autograd Function, refiner), ``scenes`` (seeded synthetic inputs), ``build``
(in-tree nvcc build).  Importing the package loads nothing; the first call that needs the
library loads it and fails loudly if it cannot.
"""
