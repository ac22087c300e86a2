"""GB300 (sm_103a) renderer for the simplified, two-parameter Fuzzy Metaballs model
("Flexible Techniques for Differentiable Rendering with 3D Gaussians", Keselman &
Hebert, WACV 2024): per-pixel depth, alpha, blended normal and optical flow from K
3D Gaussians, with a hand-written adjoint.

Submodules:
  fmb       -- ctypes binding of libfmb.so (include/fmb.h), the Renderer, the
               torch.autograd wrapper and the 6-DoF pose-gradient helper
  pipeline  -- host-fed steps with copies overlapped across steps (HostPipeline)
  step      -- reconstruction step (render, loss, adjoint, Adam) in one CUDA graph
  autotune  -- tile autotuner with a per-layout cache
  split     -- Sec. 8 split / remove criteria and the split itself (host)
  shard     -- view sharding over ranks and the gradient all-reduce
  probe     -- FP32 / MUFU throughput probe
  synth     -- seeded synthetic scenes (inputs only)
  build     -- nvcc build of libfmb.so
"""

__version__ = "0.1.0"
