"""Batched training step over many views (forward, HDR loss, backward) as one
captured CUDA graph, and the plain one-view-per-call path it is compared with.

The paper renders and optimises every cache level separately and names a
joint rasterisation of several Gaussian sets as future work (Sec. 5); here
all views of all scenes go through one binning and ONE persistent launch
that renders every view, evaluates its HDR loss and differentiates it
(``gsc_train_batch``), and the whole step -- gradient clears, the launch,
the per-view loss reductions -- replays from a CUDA graph, so the host issues
one call per step.  ``step_separate`` is the same step with the forward, the
losses and the backward as separate launches (``gsc_render_batch``).
"""
from __future__ import annotations

import numpy as np
import torch

from . import gsc, synth

RESOLUTIONS = ((256, 256), (640, 480), (1280, 720), (1920, 1080))


def uneven_views(n_views: int, n_scenes: int, seed: int):
    """(scene index, camera) pairs: view v shows scene v mod n_scenes from orbit
    angle 11.25 v degrees at a resolution drawn from RESOLUTIONS."""
    rng = np.random.default_rng(seed)
    out = []
    for v in range(n_views):
        w, h = RESOLUTIONS[int(rng.integers(0, len(RESOLUTIONS)))]
        out.append((v % n_scenes, synth.orbit_camera(w, h, 11.25 * v)))
    return out


class BatchedStep:
    """Forward + HDR loss + backward of all views; the gradients of views of
    the same scene accumulate into that scene's buffer."""

    def __init__(self, scenes, views, cfg: gsc.RasterCfg, max_pairs: int | None = None, seed: int = 7,
                 device: str = "cuda"):
        self.scenes = scenes                      # list of (N, 16) parameter tensors
        self.cfg = cfg
        self.grads = [torch.zeros_like(p) for p in scenes]
        self.views = []
        total = 0
        max_w = max_h = 1
        for k, (si, cam) in enumerate(views):
            c = gsc.camera(cam)
            h, w = c.height, c.width
            max_w, max_h = max(max_w, w), max(max_h, h)
            total += scenes[si].shape[0]
            target = torch.from_numpy(synth.uniform_image(3, h, w, seed + k)).to(device)
            self.views.append(dict(params=scenes[si], cam=c, scene=si, grads=self.grads[si],
                                   image=torch.zeros((3, h, w), device=device),
                                   dL_dimage=torch.zeros((3, h, w), device=device), target=target))
        self.losses = torch.zeros(len(self.views), device=device)
        for k, v in enumerate(self.views):
            v["loss"] = self.losses[k]
        if max_pairs is None:
            px = sum(v["cam"].width * v["cam"].height for v in self.views) / len(self.views)
            # per-view bins (bin_size 0) go down to 32 px on the small views
            max_pairs = int(min((1 << 31) - 1, total * max(24.0, 96.0 * px / (1920 * 1080))))
        self.ws = gsc.Workspace(total, max_pairs, max_w, max_h, device, max_views=len(self.views))
        self.graph = None

    def _zero_grads(self, stream):
        # the clears run on the stream the batch runs on, so they are ordered before its atomics
        with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
            for g in self.grads:
                g.zero_()

    def step(self, stream=None):
        self._zero_grads(stream)
        gsc.train_batch(self.views, self.cfg, self.ws, gsc.LOSS_HDR, stream=stream)

    def step_separate(self, stream=None):
        self._zero_grads(stream)
        gsc.render_batch(self.views, gsc.BATCH_FWD, self.cfg, self.ws, stream=stream)
        for v in self.views:
            gsc.loss(gsc.LOSS_HDR, v["image"], v["target"], self.ws, dL_dpred=v["dL_dimage"], loss_out=v["loss"],
                     stream=stream)
        gsc.render_batch(self.views, gsc.BATCH_BWD, self.cfg, self.ws, stream=stream)

    def tune(self, tiles=((16, 16), (8, 8), (32, 8), (8, 32), (16, 8)), ppts=(1, 2, 4), caps=(128, 256), bins=(0,),
             reps: int = 2):
        """Pick the fastest launch configuration for this batch (results do not
        depend on it); returns [(config dict, ms)]."""
        from . import autotune
        trials = []
        for tile, b, cap, q in autotune.candidates(tiles, bins, caps, ppts):
            self.cfg = gsc.raster_cfg(tile=tile, list_capacity=cap, bin_size=b, pixels_per_thread=q)
            self.step()
            self.ws.status()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                self.step()
            e1.record()
            e1.synchronize()
            self.ws.status()
            trials.append((dict(tile=list(tile), bin=b, list_capacity=cap, pixels_per_thread=q),
                           e0.elapsed_time(e1) / reps))
        best = min(trials, key=lambda t: t[1])[0]
        self.cfg = gsc.raster_cfg(tile=best["tile"], list_capacity=best["list_capacity"], bin_size=best["bin"],
                                  pixels_per_thread=best["pixels_per_thread"])
        return trials

    def capture(self):
        """Warm up eagerly on a side stream, then capture one step."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.ws.status()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=s):
            self.step()
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()

    def plain_step(self, ws: gsc.Workspace, stream=None):
        """The same work one view per call: render, loss, backward."""
        for g in self.grads:
            g.zero_()
        for v in self.views:
            gsc.cache_render(v["params"], v["cam"], self.cfg, ws, image=v["image"], stream=stream)
            gsc.loss(gsc.LOSS_HDR, v["image"], v["target"], ws, dL_dpred=v["dL_dimage"], loss_out=v["loss"],
                     stream=stream)
            gsc.cache_backward(v["params"], v["cam"], self.cfg, ws, v["dL_dimage"], v["grads"], stream=stream)
