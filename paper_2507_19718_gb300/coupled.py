"""Cache-coupled tracing: how the cache sampling coefficient C of Algorithm 1
(with the natural-termination cache sampling and the Eq. 2 correction) moves
the tracer along the bias-variance and runtime trade-off (Sec. 3.4, Sec. 4.3
"Visual Quality", Sec. 4.4 "Performance").

A cache is trained at the paper's C = 0.5 from a fixed view; then, for every
C of the sweep, the same cache feeds ``eval_frames`` independent 1-spp traces
(no training), timed with CUDA events.  ``tr_out`` picks the reading of
Algorithm 1's Tr_out for the training and the sweep (cumulative, or per call
as the algorithm is printed).  Against a reference traced without
the cache at ``ref_spp`` samples per pixel, each C yields the squared bias of
the mean image (less the variance the mean still carries), the per-pixel
variance across frames and their sum (MSE of one frame).  "off" is the
tracer without the cache.  Every step is a call of the C ABI.
"""
from __future__ import annotations

import numpy as np
import torch

from . import gsc, synth
from .frame import FrameLoop

C_SWEEP = (0.05, 0.1, 0.25, 0.5, 1.0, 2.0, 4.0)


def sweep(scene: synth.Scene, level_sizes, width: int = 480, height: int = 270, Cs=C_SWEEP,
          train_frames: int = 48, eval_frames: int = 24, ref_spp: int = 256, max_bounces: int = 8,
          angle: float = 20.0, seed: int = synth.BASE_SEED + 31, device: str = "cuda",
          tr_out: int = gsc.TR_OUT_PER_CALL):
    cam = gsc.camera(synth.orbit_camera(width, height, angle))
    loop = FrameLoop(scene, level_sizes, width, height, spp=1, max_bounces=max_bounces, seed=seed, C_term=0.5,
                     device=device, tr_out=tr_out)
    for f in range(train_frames):
        loop.frame(cam, f)
    K = loop.K
    # reference: the same view traced without the cache
    _, ref = gsc.trace(loop.scene, cam, ref_spp, max_bounces, K, seed + 1, 1 << 20)
    ref = ref.double()
    # the cache as trained, rendered once
    loop.render_levels(cam)
    cache = loop.renders.clone()
    targets = torch.empty_like(loop.targets)
    img = torch.empty_like(loop.image)
    rows = []
    runs = [("off", None)] + [(c, c) for c in Cs]
    for label, c in runs:
        acc = torch.zeros_like(ref)
        acc2 = torch.zeros_like(ref)
        ms = 0.0
        for f in range(eval_frames):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gsc.trace(loop.scene, cam, 1, max_bounces, K, seed + 2, 10_000 + f, C_term=c or 0.0,
                      cache=cache if c else None, targets=targets, image=img, tr_out=tr_out)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            x = img.double()
            acc += x
            acc2 += x * x
        mean = acc / eval_frames
        var = (acc2 / eval_frames - mean * mean).clamp_min(0) * eval_frames / max(eval_frames - 1, 1)
        variance = float(var.mean())
        if label == "off":
            var_ref = variance / ref_spp  # the reference is the uncached tracer at ref_spp samples
        # the mean of eval_frames frames still carries variance / eval_frames, the reference var_ref
        bias2 = max(float(((mean - ref) ** 2).mean()) - variance / eval_frames - var_ref, 0.0)
        rows.append({"C": label, "trace_ms": round(ms / eval_frames, 4), "bias2": bias2, "variance": variance,
                     "mse_per_frame": bias2 + variance})
    return rows
