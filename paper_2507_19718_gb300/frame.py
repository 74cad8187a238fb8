"""One GSCache frame on the GPU (Sec. 3.1, Fig. 4): the path tracer produces
the K intermediate path buffers, then every cache level is rendered,
compared with its buffer by the HDR loss, differentiated and stepped by AdamW
with the viewport-adaptive learning rate of Eq. 4.

Every step is a call of the C ABI (``gsc``); this module only sequences the
calls and owns the device tensors.
"""
from __future__ import annotations

import copy
import ctypes as C

import numpy as np
import torch

from . import gsc, synth


class CacheLevel:
    """Parameters, gradients and Adam moments of one cache level (N x 16 FP32).
    With ``store`` (four tensors of a larger parameter set and the row
    offset) the level's tensors are views into it."""

    def __init__(self, params: np.ndarray, device="cuda", store=None):
        if store is None:
            self.params = torch.from_numpy(np.ascontiguousarray(params, np.float32)).to(device)
            self.grads = torch.zeros_like(self.params)
            self.m = torch.zeros_like(self.params)
            self.v = torch.zeros_like(self.params)
        else:
            (P, G, M, V), r0 = store
            r1 = r0 + params.shape[0]
            self.params, self.grads, self.m, self.v = P[r0:r1], G[r0:r1], M[r0:r1], V[r0:r1]
            self.params.copy_(torch.from_numpy(np.ascontiguousarray(params, np.float32)))

    @property
    def n(self) -> int:
        return self.params.shape[0]


class FrameLoop:
    """Path-trace targets, then train and render a multi-level cache, per frame.

    ``fused`` (default) renders and differentiates all K levels as one batch
    (one binning and one persistent launch per direction over all levels,
    Sec. 5's joint rasterisation of the level sets) and steps all levels with
    one AdamW launch over their contiguous parameter store; otherwise every
    level goes through its own calls.

    ``fused_train`` (default, with ``fused``): when the tracer does not read
    the cache images (C <= 0), a frame is trace -> one training step that
    renders every level, evaluates the HDR loss against its buffer and
    differentiates in the same launch, then turns the 2D gradients into
    parameter gradients and takes the AdamW step in one more kernel
    (gsc_train_step).  The rendered images are the same bits as a separate
    forward."""

    def __init__(self, scene: synth.Scene, level_sizes, width: int, height: int, spp: int = 1,
                 max_bounces: int = 8, seed: int = synth.BASE_SEED, tile=(16, 16), list_capacity: int = 256,
                 max_pairs: int | None = None, weight_decay: float = 0.01, lr=None, device: str = "cuda",
                 gaussian_seed: int | None = None, C_term: float = 0.0, bin_size: int = 0, fused: bool = True,
                 fused_train: bool = True, tr_out: int = gsc.TR_OUT_PER_CALL):
        self.width, self.height = width, height
        self.spp, self.max_bounces, self.seed = spp, max_bounces, seed
        self.K = len(level_sizes)
        self.C_term = C_term
        # reading of Algorithm 1's Tr_out when C_term > 0: per call, as the
        # algorithm is printed (it reproduces the paper's bias-variance shape)
        self.tr_out = tr_out
        self.fused = fused
        self.fused_train = fused and fused_train
        self.scene = gsc.Scene.from_synth(scene, device)
        gs = seed + 1000 if gaussian_seed is None else gaussian_seed
        total = int(sum(level_sizes))
        f32 = dict(dtype=torch.float32, device=device)
        # one contiguous parameter store; level k owns rows [off_k, off_k + N_k)
        self.store = tuple(torch.zeros((total, 16), **f32) for _ in range(4))
        self.levels = []
        off = 0
        for k, n in enumerate(level_sizes):
            self.levels.append(CacheLevel(synth.gaussians(n, gs + k), device, store=(self.store, off)))
            off += n
        n_ws = total if fused else max(level_sizes)
        if max_pairs is None:
            # log-normal scales (N(-3, 0.5)) make the large Gaussians dominate:
            # at 1080p a Gaussian's support spans ~300 px, i.e. ~33 bins of
            # 64 px; keep headroom and scale with the pixel count and bin area
            b = bin_size or 64
            per = 96.0 * (width * height) / (1920 * 1080) * (64.0 / b) ** 2
            max_pairs = int(min((1 << 31) - 1, max(1 << 16, n_ws * max(per, 4.0))))
        self.ws = gsc.Workspace(n_ws, max_pairs, width, height, device, max_views=self.K if fused else 1)
        self.cfg = gsc.raster_cfg(tile=tile, list_capacity=list_capacity, bin_size=bin_size)
        self.cfg_bwd = None  # backward launch configuration, if different from cfg
        self.lr = np.asarray(gsc.PAPER_LR if lr is None else lr, np.float32)
        self.weight_decay = weight_decay
        self.targets = torch.zeros((self.K, 3, height, width), **f32)
        self.image = torch.zeros((3, height, width), **f32)
        self.renders = torch.zeros((self.K, 3, height, width), **f32)
        self.dL = torch.zeros((self.K, 3, height, width), **f32)
        self.losses = torch.zeros((self.K,), **f32)
        self.adam_step = 0
        self.static_frames = 0
        self._last_pose = None
        self._copy_stream = None
        self._adapt = None

    def snapshot(self):
        """Copy of the training state (parameters, moments, step, schedule,
        and the state of the adaptive launch choice)."""
        P, _, M, V = self.store
        sel = copy.deepcopy(self._adapt["sel"]) if self._adapt is not None else None
        return (P.clone(), M.clone(), V.clone()), self.adam_step, self.static_frames, self._last_pose, sel

    def restore(self, snap):
        (p, m, v), self.adam_step, self.static_frames, self._last_pose, sel = snap
        P, G, M, V = self.store
        P.copy_(p)
        M.copy_(m)
        V.copy_(v)
        G.zero_()
        if self._adapt is not None and sel is not None:
            self._adapt["pending"] = []          # times of steps from before the snapshot's state
            self._adapt["sel"] = copy.deepcopy(sel)
            self.cfg_bwd = self._adapt["cfgs"][sel.current]

    def _schedule(self, c: gsc.Camera) -> float:
        """Eq. 4: frames the viewport has been unchanged (pose compared bit for bit)."""
        pose = bytes(c)
        self.static_frames = self.static_frames + 1 if pose == self._last_pose else 1
        self._last_pose = pose
        return gsc.lr_scale(self.static_frames)

    def trace(self, c: gsc.Camera, frame: int, stream=None):
        cache = self.renders if self.C_term > 0 else None
        gsc.trace(self.scene, c, self.spp, self.max_bounces, self.K, self.seed, frame, C_term=self.C_term,
                  cache=cache, targets=self.targets, image=self.image, stream=stream, tr_out=self.tr_out)

    def render_levels(self, c: gsc.Camera, stream=None):
        if self.fused:
            views = [dict(params=L.params, cam=c, image=self.renders[k]) for k, L in enumerate(self.levels)]
            gsc.render_batch(views, gsc.BATCH_FWD, self.cfg, self.ws, stream=stream)
            return
        for k, L in enumerate(self.levels):
            gsc.cache_render(L.params, c, self.cfg, self.ws, image=self.renders[k], stream=stream)

    def train_levels(self, c: gsc.Camera, lr_scale: float, stream=None):
        self.adam_step += 1
        adam = gsc.adam_params(self.lr, weight_decay=self.weight_decay, lr_scale=lr_scale, step=self.adam_step)
        cfg_b = self.cfg_bwd or self.cfg
        for k in range(self.K):
            gsc.loss(gsc.LOSS_HDR, self.renders[k], self.targets[k], self.ws, dL_dpred=self.dL[k],
                     loss_out=self.losses[k], stream=stream)
        if self.fused:
            views = [dict(params=L.params, cam=c, dL_dimage=self.dL[k], grads=L.grads)
                     for k, L in enumerate(self.levels)]
            gsc.render_batch(views, gsc.BATCH_BWD, cfg_b, self.ws, stream=stream)
            # every level has the same per-slot rates and schedule: one launch
            gsc.cache_step(*self.store, adam, stream=stream)
            return
        for k, L in enumerate(self.levels):
            gsc.cache_backward(L.params, c, cfg_b, self.ws, self.dL[k], L.grads, stream=stream)
            gsc.cache_step(L.params, L.grads, L.m, L.v, adam, stream=stream)

    def adapt_train_launch(self, cfgs, explore_every: int = 6, prior=None):
        """Choose the training step's launch configuration among ``cfgs``
        while the cache trains (``autotune.OnlineSelector``; the first is the
        starting choice): every frame's training step is timed on the device
        and every ``explore_every``-th frame runs another candidate (``prior``:
        the candidates' times if known, e.g. from the autotuner).  The
        configuration changes no result beyond the order of the FP32 sums.
        It applies to the one-launch training step (C <= 0); the separate
        launches of a cache-reading frame keep ``cfg_bwd``."""
        from .autotune import OnlineSelector
        cfgs = list(cfgs)
        self._adapt = dict(cfgs=cfgs, sel=OnlineSelector(len(cfgs), explore_every, prior=prior), pending=[],
                           pool=[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                                 for _ in range(3)], slot=0)
        self.cfg_bwd = cfgs[0]
        return self._adapt["sel"]

    def _adapt_collect(self, lag: int):
        """Report the timed training steps that have finished; wait for the
        oldest ones until at most ``lag`` remain in flight (the frames queued
        behind them keep the device busy meanwhile)."""
        a = self._adapt
        while len(a["pending"]) > lag:
            i, e0, e1 = a["pending"].pop(0)
            e1.synchronize()
            a["sel"].report(i, e0.elapsed_time(e1))
        while a["pending"] and a["pending"][0][2].query():
            i, e0, e1 = a["pending"].pop(0)
            a["sel"].report(i, e0.elapsed_time(e1))

    def train_step(self, c: gsc.Camera, lr_scale: float, stream=None):
        """Render + HDR loss + backward of all levels in one launch, the
        per-Gaussian gradients and the AdamW step in one more (gsc_train_step)."""
        self.adam_step += 1
        adam = gsc.adam_params(self.lr, weight_decay=self.weight_decay, lr_scale=lr_scale, step=self.adam_step)
        # no gradient is accumulated between frames, so none is passed
        views = [dict(params=L.params, cam=c, target=self.targets[k], image=self.renders[k], loss=self.losses[k],
                      m=L.m, v=L.v) for k, L in enumerate(self.levels)]
        a = self._adapt
        if a is None:
            gsc.train_step(views, adam, self.cfg_bwd or self.cfg, self.ws, gsc.LOSS_HDR, stream=stream)
            return
        # the choice for this frame sees the times of the frames before the
        # previous one; the previous frame's work keeps the device busy while
        # the host waits for them
        self._adapt_collect(lag=1)
        i = a["sel"].choose()
        self.cfg_bwd = a["cfgs"][a["sel"].current]
        e0, e1 = a["pool"][a["slot"]]
        a["slot"] = (a["slot"] + 1) % len(a["pool"])
        s = torch.cuda.current_stream() if stream is None else stream
        e0.record(s)
        gsc.train_step(views, adam, a["cfgs"][i], self.ws, gsc.LOSS_HDR, stream=stream)
        e1.record(s)
        a["pending"].append((i, e0, e1))

    def frame(self, cam, frame: int, stream=None):
        """One frame: render the cache (its images feed the tracer when C > 0),
        trace the targets, then train every level on its buffer."""
        c = cam if isinstance(cam, gsc.Camera) else gsc.camera(cam)
        lr_scale = self._schedule(c)
        if self.fused_train and self.C_term <= 0:
            self.trace(c, frame, stream)
            self.train_step(c, lr_scale, stream)
            return self.losses
        self.render_levels(c, stream)
        self.trace(c, frame, stream)
        self.train_levels(c, lr_scale, stream)
        return self.losses

    def frame_to_host(self, cam, frame: int, host_image: torch.Tensor, host_losses: torch.Tensor, stream=None):
        """``frame`` with its results read back to host memory (pinned, for the
        copies to be asynchronous): the display image is final once the tracer
        has run, so it is copied on a side stream while the levels train; the
        level losses follow the step.  Both host tensors are complete once
        ``stream`` (default: the current stream) is synchronised, and the next
        frame's tracer, which rewrites the image, runs after the copy."""
        s = torch.cuda.current_stream() if stream is None else stream
        if not (self.fused_train and self.C_term <= 0):
            # the image depends on this frame's cache render: nothing to overlap
            self.frame(cam, frame, s)
            with torch.cuda.stream(s):
                host_image.copy_(self.image, non_blocking=True)
                host_losses.copy_(self.losses, non_blocking=True)
            return host_losses
        if self._copy_stream is None:
            self._copy_stream = torch.cuda.Stream(device=self.image.device)
        c = cam if isinstance(cam, gsc.Camera) else gsc.camera(cam)
        lr_scale = self._schedule(c)
        self.trace(c, frame, s)
        traced = torch.cuda.Event()
        traced.record(s)
        cs = self._copy_stream
        cs.wait_event(traced)
        with torch.cuda.stream(cs):
            host_image.copy_(self.image, non_blocking=True)
        read = torch.cuda.Event()
        read.record(cs)
        self.train_step(c, lr_scale, s)
        with torch.cuda.stream(s):
            host_losses.copy_(self.losses, non_blocking=True)
        s.wait_event(read)
        return host_losses
