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



def drift_candidates(best: Trial, trials, k: int = 2):
    """Candidates of an online choice for a training step tuned as ``best``:
    ``best`` first, then the fastest trial at each of the ``k`` next lower
    pixels-per-thread values (the direction the choice drifts as a cache
    trains); with no lower value, the fastest at the next higher one."""
    lower = sorted({t.ppt for t in trials if t.ppt < best.ppt}, reverse=True)[:k]
    if not lower:
        lower = sorted({t.ppt for t in trials if t.ppt > best.ppt})[:1]
    return [best] + [min((t for t in trials if t.ppt == q), key=lambda t: t.ms) for q in lower]

class OnlineSelector:
    """Launch configuration of a step that repeats while its best choice
    drifts with the data.  In the training step of a cache the pixels of a
    tile stop at more and more different depths as the cache trains, and
    fewer pixels per thread start to win (at 1080p with 1M Gaussians: 4 per
    thread fastest on the first frames, 2 per thread 27% faster than 4 after
    25 frames of an orbiting camera).

    Every step runs exactly once with one configuration, so nothing is added
    to the work: the current choice runs on most steps and every
    ``explore_every``-th step runs the next other candidate in turn.  The
    current choice's time is a running mean (weight ``alpha`` on the newest
    step), another candidate's time is its newest measurement; the selector
    moves to a candidate that is faster by more than ``margin``.  When the
    current choice's time rises more than ``drift`` above its lowest since it
    was chosen (the data changed), the next steps explore every other
    candidate at once.  An exploration step costs the candidate's whole gap
    (at 1080p one pixel per thread runs 35-55% behind four on every frame of
    the drift, two per thread about 20% on the first 20 frames), and a
    drift is gradual, so a regular round skips a candidate until
    1 + gap / ``gap_step`` rounds (at most ``far_every``) have passed since it
    last ran, gap being its newest time over the current choice's, less 1;
    a candidate never measured runs at the first round, and the rounds a
    drift starts run every candidate.  ``prior`` (optional, one
    time per candidate, None or NaN where unknown) seeds the other
    candidates' times, e.g. from the autotuner's trials.  Times
    come back through ``report`` whenever they are known (a step's device
    time is read without waiting for it)."""

    def __init__(self, n: int, explore_every: int = 4, alpha: float = 0.25, margin: float = 0.03,
                 drift: float = 0.05, gap_step: float = 0.05, far_every: int = 8, prior=None):
        if n < 1 or explore_every < 2 or far_every < 1:
            raise ValueError("need at least one candidate, explore_every >= 2 and far_every >= 1")
        if prior is not None and len(prior) != n:
            raise ValueError("prior needs one entry per candidate")
        self.n, self.explore_every, self.alpha, self.margin, self.drift = n, explore_every, alpha, margin, drift
        self.gap_step, self.far_every = gap_step, far_every
        self.current = 0
        self.est = [None] * n
        if prior is not None:
            for j in range(1, n):
                if prior[j] is not None and prior[j] == prior[j]:  # NaN: unknown
                    self.est[j] = float(prior[j])
        self._rounds = 0          # regular exploration rounds so far
        self._last = [None] * n   # round in which each candidate last ran
        self.runs = [0] * n
        self.switches = 0
        self._step = 0
        self._next = 0
        self._low = None          # lowest time of the current choice since it was chosen
        self._burst = 0           # steps left that explore at once

    def choose(self) -> int:
        """Index of the candidate for the next step."""
        self._step += 1
        i = self.current
        if self.n > 1 and (self._burst > 0 or self._step % self.explore_every == 0):
            burst = self._burst > 0
            self._burst = max(0, self._burst - 1)
            self._step = 0            # the next regular exploration counts from here
            if not burst:
                self._rounds += 1
            nxt = self._next
            for _ in range(self.n):
                nxt = (nxt + 1) % self.n
                if nxt != self.current and (burst or self._due(nxt)):
                    i = self._next = nxt
                    self._last[i] = self._rounds
                    break
        self.runs[i] += 1
        return i

    def _due(self, j: int) -> bool:
        """Whether candidate j's next regular exploration is due."""
        cur, e = self.est[self.current], self.est[j]
        if cur is None or e is None:
            return True
        gap = max(0.0, e / cur - 1.0)
        wait = min(self.far_every, 1 + int(gap / self.gap_step + 1e-6))
        last = self._last[j] if self._last[j] is not None else 0  # a prior counts from the start
        return self._rounds - last >= wait

    def report(self, i: int, ms: float):
        """Device time of a step that ran candidate ``i``."""
        if i == self.current and self.est[i] is not None:
            self.est[i] += self.alpha * (ms - self.est[i])
        else:
            self.est[i] = ms
        cur = self.est[self.current]
        if cur is None:
            return
        if i == self.current:
            if self._low is None or cur < self._low:
                self._low = cur
            elif cur > self._low * (1.0 + self.drift):
                self._burst = self.n - 1
                self._low = cur
        best = min((j for j in range(self.n) if self.est[j] is not None), key=lambda j: self.est[j])
        if best != self.current and self.est[best] < cur * (1.0 - self.margin):
            self.current = best
            self.switches += 1
            self._low = self.est[best]
