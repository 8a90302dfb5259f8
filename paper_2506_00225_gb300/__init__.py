"""GB300-native semantic Gaussian-splatting rasterizer (ActiveSGM hot path).

Importing the package is cheap: the native library is loaded on first use by
``paper_2506_00225_gb300.raster`` (which fails loudly when it is missing).

Modules:
  scenes  -- seeded synthetic scenes and cameras (inputs only)
  build   -- in-tree nvcc build of libgs.so for sm_103a
  _native -- ctypes declarations of include/gs.h
  raster  -- PyTorch layer: workspace, autograd Function, candidates, L1 loss
"""
__all__ = ["scenes", "build", "raster"]
