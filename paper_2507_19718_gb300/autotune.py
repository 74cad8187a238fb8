"""Autotuner of the rasterizer launch configuration.

The tile shape, the coarse bin size and the shared-memory staging capacity
never change a result bit (every pixel composites the same ordered list);
they only change speed.  ``autotune`` times the render and its backward for
each candidate through the C ABI (CUDA events on the launching stream) on the
caller's actual levels and camera, and returns the fastest configuration.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import torch

from . import gsc

TILES = ((16, 16), (8, 8), (32, 8), (16, 8), (8, 16))
BINS = (32, 64, 128)
CAPS = (96, 128, 256, 512)
PPTS = (1, 2, 4, 8)
# (tile, pixels per thread) pairs the library is compiled for
COMPILED = {1: {(16, 16), (8, 8), (32, 8), (16, 8), (8, 16), (8, 32), (32, 4)},
            2: {(16, 16), (32, 8), (16, 8), (8, 16), (8, 32)},
            4: {(16, 16), (32, 8), (8, 32)},
            8: {(16, 16), (32, 8), (8, 32)}}


@dataclass
class Trial:
    tile: tuple
    bin_size: int
    list_capacity: int
    ppt: int
    ms: float

    def cfg(self, **kw) -> gsc.RasterCfg:
        return gsc.raster_cfg(tile=self.tile, list_capacity=self.list_capacity, bin_size=self.bin_size,
                              pixels_per_thread=self.ppt, **kw)


def candidates(tiles=TILES, bins=BINS, caps=CAPS, ppts=PPTS):
    for t, b, c, q in itertools.product(tiles, bins, caps, ppts):
        if b % t[0] or b % t[1] or c < t[0] * t[1] // q or tuple(t) not in COMPILED.get(q, ()):
            continue
        yield t, b, c, q


def time_config(levels, cam, ws: gsc.Workspace, tile, bin_size, cap, ppt=1, backward=True, reps=2, stream=None,
                fused=False, forward=True, train=False):
    """Mean ms of rendering (and/or differentiating) every level once; with
    ``fused`` all levels go through one batched call per direction; with
    ``train`` all levels go through one training step (gsc_train_batch)."""
    c = cam if isinstance(cam, gsc.Camera) else gsc.camera(cam)
    cfg = gsc.raster_cfg(tile=tile, list_capacity=cap, bin_size=bin_size, pixels_per_thread=ppt)
    dev = levels[0].device
    imgs = [torch.empty((3, c.height, c.width), dtype=torch.float32, device=dev) for _ in levels]
    dl = torch.full((3, c.height, c.width), 1e-3, dtype=torch.float32, device=dev)
    grads = [torch.zeros_like(p) for p in levels]
    views = [dict(params=p, cam=c, image=im, dL_dimage=dl, grads=g) for p, im, g in zip(levels, imgs, grads)]
    s = torch.cuda.current_stream() if stream is None else stream
    if train:
        losses = torch.zeros(len(levels), dtype=torch.float32, device=dev)
        tviews = [dict(params=p, cam=c, target=dl, image=im, grads=g, loss=losses[k])
                  for k, (p, im, g) in enumerate(zip(levels, imgs, grads))]

    def once():
        if train:
            gsc.train_batch(tviews, cfg, ws, gsc.LOSS_HDR, stream=s)
            return
        if fused:
            if forward:
                gsc.render_batch(views, gsc.BATCH_FWD, cfg, ws, stream=s)
            if backward:
                gsc.render_batch(views, gsc.BATCH_BWD, cfg, ws, stream=s)
            return
        for v in views:
            if forward:
                gsc.cache_render(v["params"], c, cfg, ws, image=v["image"], stream=s)
            if backward:
                gsc.cache_backward(v["params"], c, cfg, ws, dl, v["grads"], stream=s)

    once()  # warm-up
    ws.status(s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        once()
    e1.record(s)
    e1.synchronize()
    ws.status(s)
    return e0.elapsed_time(e1) / reps


def autotune(levels, cam, ws: gsc.Workspace, backward=True, cands=None, reps=2, verbose=False, fused=False,
             forward=True, train=False):
    """Fastest (tile, bin, capacity, pixels per thread) for rendering and/or
    differentiating the given levels from `cam`.  Returns (best Trial, all
    trials)."""
    trials = []
    for tile, b, cap, q in (cands if cands is not None else candidates()):
        ms = time_config(levels, cam, ws, tile, b, cap, q, backward=backward, reps=reps, fused=fused,
                         forward=forward, train=train)
        trials.append(Trial(tile, b, cap, q, ms))
        if verbose:
            print(f"tile {tile[0]}x{tile[1]} bin {b} cap {cap} ppt {q}: {ms:.3f} ms", flush=True)
    best = min(trials, key=lambda t: t.ms)
    return best, trials
