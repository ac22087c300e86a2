"""GB300 (sm_103a) renderer for the simplified, two-parameter Fuzzy Metaballs model
("Flexible Techniques for Differentiable Rendering with 3D Gaussians", Keselman &
Hebert, WACV 2024): per-pixel depth, alpha, blended normal and optical flow from K
3D Gaussians, with a hand-written adjoint.

Submodules:
  fmb    -- ctypes binding of libfmb.so (include/fmb.h) and torch.autograd wrapper
  synth  -- seeded synthetic scenes (inputs only)
  build  -- nvcc build of libfmb.so
"""

__version__ = "0.1.0"
