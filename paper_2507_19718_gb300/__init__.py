"""GB300-native (sm_103a) implementation of the GSCache hot path.

GSCache (Bauer, Wu, Gadirov, Ma) caches path-space radiance of a volume path
tracer in multi-level sets of 3D Gaussians that are splatted every frame and
trained on the fly against the tracer's per-path-length target buffers.

Modules:
  gsc    -- Python binding of the C-ABI CUDA library (include/gsc.h) and the
            autograd wrapper of the cache render
  frame  -- the per-frame loop (trace, render, loss, backward, AdamW)
  synth  -- seeded synthetic inputs (no method arithmetic)
  build  -- in-tree nvcc build of the CUDA library
"""
from . import synth  # noqa: F401

__all__ = ["synth"]
