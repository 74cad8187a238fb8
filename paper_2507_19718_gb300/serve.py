"""Serving loop of a GSCache deployment: resident scenes, continuous batching
of view requests, transfer-function changes that retrain the cache on the
fly, and p50/p99 frame latency.

A view request asks for the cache images of one scene (every level, the
images the path tracer reads, Sec. 3.1) at a camera pose and resolution.  A
transfer-function change replaces the scene's TF (the event the paper's cache
is designed to adapt to, Sec. 1 and 4.4), resets the learning-rate schedule of
Eq. 4 and retrains the cache for a fixed number of frames.

Requests that arrive while others are on the GPU are admitted into the next
batch as soon as a batch slot, a workspace and HBM budget are free; up to two
view batches are in flight on the render stream and retraining frames run on
their own stream, so the work of different requests overlaps on the device.
Every step is a call of the C ABI.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import gsc, synth
from .frame import CacheLevel

VIEW_RESOLUTIONS = ((256, 256), (640, 480), (1280, 720), (1920, 1080))


@dataclass
class Request:
    rid: int
    kind: str                 # "view" or "tf"
    scene: int
    arrival: float            # seconds after the start of the trace
    angle: float = 0.0        # orbit angle of a view request
    width: int = 0
    height: int = 0
    tf_seed: int = 0          # seed of a new 8-point TF
    done: float = float("nan")
    images: list = field(default_factory=list)


def poisson_trace(rate: float, duration: float, n_scenes: int, seed: int, tf_fraction: float = 0.1,
                  resolutions=VIEW_RESOLUTIONS):
    """Poisson arrivals: view requests at the given resolutions, a fraction of
    transfer-function changes."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        scene = int(rng.integers(0, n_scenes))
        if rng.uniform() < tf_fraction:
            out.append(Request(len(out), "tf", scene, t, tf_seed=int(rng.integers(0, 1 << 30))))
        else:
            w, h = resolutions[int(rng.integers(0, len(resolutions)))]
            out.append(Request(len(out), "view", scene, t, angle=float(rng.uniform(0, 360)), width=w, height=h))
    return out


class ResidentScene:
    """A scene kept on the device: volume, tracer handle, and a multi-level
    cache with its optimiser state and learning-rate schedule."""

    def __init__(self, scene: synth.Scene, level_sizes, seed: int, device="cuda"):
        self.desc = scene
        self.handle = gsc.Scene.from_synth(scene, device)
        self.levels = [CacheLevel(synth.gaussians(n, seed + k), device) for k, n in enumerate(level_sizes)]
        self.adam_step = 0
        self.static_frames = 0
        self.retrain_left = 0
        self.frames_trained = 0

    @property
    def n_gaussians(self) -> int:
        return sum(L.n for L in self.levels)

    def set_tf(self, tf_seed: int):
        pos, rgba = synth.transfer_function(8, tf_seed)
        self.handle.set_tf(pos, rgba)

    def state_bytes(self) -> int:
        return int(self.handle.density.numel() * 4 + sum(L.params.numel() * 4 * 4 for L in self.levels))


class Trainer:
    """Retraining frames of one scene at a fixed training view: trace the K
    target buffers, then one training step for all levels (render, HDR loss
    and backward in one launch, the per-Gaussian gradients and AdamW in one
    more: gsc_train_step).  max_gaussians: the largest scene's total over its
    levels."""

    def __init__(self, width: int, height: int, levels: int, max_gaussians: int, cfg: gsc.RasterCfg,
                 spp: int = 1, max_bounces: int = 8, lr=None, weight_decay: float = 0.01, device="cuda"):
        self.w, self.h, self.K = width, height, levels
        self.cfg = cfg
        self.spp, self.max_bounces = spp, max_bounces
        self.lr = np.asarray(gsc.PAPER_LR if lr is None else lr, np.float32)
        self.weight_decay = weight_decay
        # bins chosen per view (bin_size 0) go down to 32 px, so a Gaussian
        # can reach a dozen bins even at training resolution
        pairs = int(max_gaussians * max(24.0, 96.0 * width * height / (1920 * 1080)))
        self.ws = gsc.Workspace(max_gaussians, pairs, width, height, device, max_views=levels)
        f32 = dict(dtype=torch.float32, device=device)
        self.targets = torch.zeros((levels, 3, height, width), **f32)
        self.image = torch.zeros((3, height, width), **f32)
        self.loss = torch.zeros((levels,), **f32)

    def tune(self, sc: "ResidentScene", tiles=((16, 16), (8, 8), (32, 8), (8, 32), (16, 8)), bins=(0, 64),
             caps=(128, 256), ppts=(1, 2, 4)):
        """Pick the fastest launch configuration of the training step at this
        resolution on scene sc (its levels trained from the training view);
        results do not depend on it.  Returns the trials."""
        from . import autotune
        cam = synth.orbit_camera(self.w, self.h, 30.0)
        cands = list(autotune.candidates(tiles, bins, caps, ppts))
        best, trials = autotune.autotune([L.params for L in sc.levels], cam, self.ws, cands=cands, reps=2,
                                         train=True)
        self.cfg = best.cfg()
        return trials

    def frame(self, sc: ResidentScene, angle: float, frame: int, seed: int, stream=None):
        c = gsc.camera(synth.orbit_camera(self.w, self.h, angle))
        sc.static_frames += 1   # the training view stays put: Eq. 4 decays
        sc.adam_step += 1
        adam = gsc.adam_params(self.lr, weight_decay=self.weight_decay,
                               lr_scale=gsc.lr_scale(sc.static_frames), step=sc.adam_step)
        gsc.trace(sc.handle, c, self.spp, self.max_bounces, self.K, seed, frame, targets=self.targets,
                  image=self.image, stream=stream)
        views = [dict(params=L.params, cam=c, target=self.targets[k], loss=self.loss[k], m=L.m, v=L.v)
                 for k, L in enumerate(sc.levels)]
        gsc.train_step(views, adam, self.cfg, self.ws, gsc.LOSS_HDR, stream=stream)
        sc.frames_trained += 1


class Server:
    """Resident scenes served by continuous batching (``run_batched``) or one
    view per call in arrival order (``run_plain``)."""

    def __init__(self, scenes, cfg: gsc.RasterCfg, hbm_budget: int | None = None, max_views: int = 32,
                 train_res=(320, 240), retrain_frames: int = 16, max_batch_gaussians: int | None = None,
                 max_res=(1920, 1080), seed: int = 99, device: str = "cuda", keep_images: bool = False,
                 train_cfg: gsc.RasterCfg | None = None):
        self.scenes = scenes
        self.keep_images = keep_images   # completed requests keep their images (tests)
        self.cfg = cfg
        self.K = len(scenes[0].levels)
        self.max_views = max_views - max_views % self.K
        self.retrain_frames = retrain_frames
        self.seed = seed
        self.device = device
        self.max_batch_g = max_batch_gaussians or 4 * max(sc.n_gaussians for sc in scenes)
        pairs = int(min((1 << 31) - 1, self.max_batch_g * 24))
        self.view_ws = [gsc.Workspace(self.max_batch_g, pairs, max_res[0], max_res[1], device,
                                      max_views=self.max_views) for _ in range(2)]
        self.plain_ws = gsc.Workspace(max(L.n for sc in scenes for L in sc.levels), pairs // 4, max_res[0],
                                      max_res[1], device)
        self.trainer = Trainer(train_res[0], train_res[1], self.K, max(sc.n_gaussians for sc in scenes),
                               train_cfg or cfg,
                               device=device)
        self.fixed_bytes = (sum(sc.state_bytes() for sc in scenes) + sum(ws.nbytes for ws in self.view_ws) +
                            self.plain_ws.nbytes + self.trainer.ws.nbytes)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = int(0.8 * free) + self.fixed_bytes   # 80% of what was free after start-up
        self.budget = hbm_budget
        self.stats = {}
        self.view_cfgs = {}   # (width, height) -> launch configuration of its views (tune_views)

    def tune_views(self, sc: "ResidentScene", resolutions=VIEW_RESOLUTIONS, tiles=((16, 16), (8, 8)),
                   bins=(0, 128), caps=(96, 256), ppts=(1, 2, 4)):
        """Pick the fastest launch configuration of a view's batched forward
        render (its K levels) at each request resolution, on scene sc.  A
        small view has few tiles for the GPU's SMs, so it wants more threads
        per tile than a 1080p one.  Results do not depend on it.  Returns
        {(width, height): trials}."""
        from . import autotune
        out = {}
        for w, h in resolutions:
            cam = synth.orbit_camera(w, h, 30.0)
            cands = list(autotune.candidates(tiles, bins, caps, ppts))
            best, trials = autotune.autotune([L.params for L in sc.levels], cam, self.view_ws[0], cands=cands,
                                             reps=2, fused=True, backward=False)
            self.view_cfgs[(w, h)] = best.cfg()
            out[(w, h)] = trials
        return out

    def _cfg_for(self, reqs) -> gsc.RasterCfg:
        """Launch configuration of a batch: the one tuned for its largest view."""
        r = max(reqs, key=lambda q: q.width * q.height)
        return self.view_cfgs.get((r.width, r.height), self.cfg)

    def _out_bytes(self, r: Request) -> int:
        return 3 * r.width * r.height * 4 * self.K

    def _train_one(self, sc: ResidentScene, stream):
        self.trainer.frame(sc, angle=30.0, frame=sc.frames_trained, seed=self.seed + 1000 * self.scenes.index(sc),
                           stream=stream)
        sc.retrain_left -= 1

    # -------------------------------------------------------------- batched

    def run_batched(self, trace):
        K, cfg = self.K, self.cfg
        pending = collections.deque(sorted(trace, key=lambda r: r.arrival))
        queue = collections.deque()
        inflight = collections.deque()        # (event, requests, workspace index, bytes)
        free_ws = list(range(len(self.view_ws)))
        # views on a higher-priority stream: when a CTA of the retraining
        # frame retires, the block scheduler hands the SM to a view's CTA first
        rs, ts = torch.cuda.Stream(priority=-1), torch.cuda.Stream(priority=0)
        tf_waiting = collections.defaultdict(list)   # scene -> TF requests completed by its retraining
        last_train_ev = {}                    # scene -> event of its last enqueued training frame
        last_render_ev = {}                   # scene -> event of its last enqueued render batch
        train_ev, train_req_scene = None, None
        in_flight_bytes, rr = 0, 0
        n_batches, views_per_batch = 0, []
        ref = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ref.record()
        t0 = time.perf_counter()

        def finish(ev, reqs):
            ev.synchronize()
            t = ref.elapsed_time(ev) / 1e3
            for r in reqs:
                r.done = t
                if not self.keep_images:
                    r.images = []     # delivered: the output memory returns to the pool

        while pending or queue or inflight or train_ev is not None or any(s.retrain_left for s in self.scenes):
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            while inflight and inflight[0][0].query():
                ev, reqs, wi, nb = inflight.popleft()
                finish(ev, reqs)
                free_ws.append(wi)
                in_flight_bytes -= nb
            # transfer-function changes are applied when they reach the head of the queue
            while queue and queue[0].kind == "tf":
                r = queue.popleft()
                sc = self.scenes[r.scene]
                sc.set_tf(r.tf_seed)
                sc.retrain_left = self.retrain_frames
                sc.static_frames = 0
                tf_waiting[r.scene].append(r)
            # admit view requests into a batch
            if free_ws and queue and queue[0].kind == "view":
                batch, views, g, nb = [], [], 0, 0
                while queue and queue[0].kind == "view":
                    r = queue[0]
                    sc = self.scenes[r.scene]
                    ob = self._out_bytes(r)
                    over = self.fixed_bytes + in_flight_bytes + nb + ob > self.budget
                    if over and (batch or inflight):
                        break   # wait for memory; a request larger than the budget goes alone when idle
                    if len(views) + K > self.max_views or g + sc.n_gaussians > self.max_batch_g:
                        break
                    queue.popleft()
                    cam = gsc.camera(synth.orbit_camera(r.width, r.height, r.angle))
                    r.images = [torch.empty((3, r.height, r.width), device=self.device) for _ in range(K)]
                    for k, L in enumerate(sc.levels):
                        views.append(dict(params=L.params, cam=cam, image=r.images[k]))
                    batch.append(r)
                    g += sc.n_gaussians
                    nb += ob
                if batch:
                    wi = free_ws.pop()
                    for s in {r.scene for r in batch}:
                        if s in last_train_ev:
                            rs.wait_event(last_train_ev[s])   # see the scene's latest trained cache
                    with torch.cuda.stream(rs):
                        gsc.render_batch(views, gsc.BATCH_FWD, self._cfg_for(batch), self.view_ws[wi])
                        ev = torch.cuda.Event(enable_timing=True)
                        ev.record(rs)
                    for s in {r.scene for r in batch}:
                        last_render_ev[s] = ev
                    inflight.append((ev, batch, wi, nb))
                    in_flight_bytes += nb
                    n_batches += 1
                    views_per_batch.append(len(views))
            # one retraining frame at a time on the training stream
            if train_ev is not None and train_ev.query():
                if self.scenes[train_req_scene].retrain_left == 0 and tf_waiting[train_req_scene]:
                    finish(train_ev, tf_waiting.pop(train_req_scene))
                train_ev = None
            if train_ev is None:
                cands = [i for i, s in enumerate(self.scenes) if s.retrain_left > 0]
                if cands:
                    si = cands[rr % len(cands)]
                    rr += 1
                    sc = self.scenes[si]
                    if si in last_render_ev:
                        ts.wait_event(last_render_ev[si])     # renders in flight still read the cache
                    with torch.cuda.stream(ts):
                        self._train_one(sc, None)
                        ev = torch.cuda.Event(enable_timing=True)
                        ev.record(ts)
                    last_train_ev[si] = ev
                    train_ev, train_req_scene = ev, si
            if not (queue and free_ws) and (train_ev is None or not train_ev.query()):
                time.sleep(0.0001)
        torch.cuda.synchronize()
        for ws in self.view_ws + [self.trainer.ws]:
            ws.status()   # raises if a binning overflowed its pair buffers
        self.stats = dict(batches=n_batches, mean_views_per_batch=float(np.mean(views_per_batch)) if views_per_batch
                          else 0.0, wall_s=time.perf_counter() - t0)
        return trace

    # -------------------------------------------------------------- plain

    def run_plain(self, trace):
        """Arrival order on one stream, one level per render call, no batching."""
        K, cfg = self.K, self.cfg
        s = torch.cuda.current_stream()
        ref = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ref.record()
        t0 = time.perf_counter()
        events = collections.deque()

        def retire(block: bool):
            while events and (block or events[0][0].query()):
                ev, r = events.popleft()
                ev.synchronize()
                r.done = ref.elapsed_time(ev) / 1e3
                if not self.keep_images:
                    r.images = []
                block = False

        for r in sorted(trace, key=lambda r: r.arrival):
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            retire(False)
            while len(events) >= 64:      # bound the work queued ahead of the GPU
                retire(True)
            sc = self.scenes[r.scene]
            if r.kind == "view":
                cam = gsc.camera(synth.orbit_camera(r.width, r.height, r.angle))
                r.images = [torch.empty((3, r.height, r.width), device=self.device) for _ in range(K)]
                for k, L in enumerate(sc.levels):
                    gsc.cache_render(L.params, cam, self._cfg_for([r]), self.plain_ws, image=r.images[k], stream=s)
            else:
                sc.set_tf(r.tf_seed)
                sc.retrain_left = self.retrain_frames
                sc.static_frames = 0
                while sc.retrain_left:
                    self._train_one(sc, s)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
            events.append((ev, r))
        torch.cuda.synchronize()
        while events:
            retire(True)
        for ws in (self.plain_ws, self.trainer.ws):
            ws.status()
        self.stats = dict(batches=len(events), mean_views_per_batch=float(K), wall_s=time.perf_counter() - t0)
        return trace


def latency_stats(trace, kind: str = "view") -> dict:
    lat = np.array([(r.done - r.arrival) * 1e3 for r in trace if r.kind == kind and r.done == r.done])
    if lat.size == 0:
        return dict(n=0)
    return dict(n=int(lat.size), p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                mean_ms=float(lat.mean()), max_ms=float(lat.max()))


def frame_scenes(n_scenes: int, base_res: int = 256, seed: int = synth.BASE_SEED + 4):
    """Eight distinct 256^3 volumes without generating eight fBm fields: the
    base blob + fBm volume rolled along a different axis and offset per scene,
    each with its own 8-point TF."""
    base = synth.scene_frame(base_res, seed=seed)
    out = []
    for k in range(n_scenes):
        dens = np.ascontiguousarray(np.roll(base.density, shift=23 * k, axis=k % 3))
        pos, rgba = synth.transfer_function(8, seed + 100 + k)
        out.append(synth.Scene(density=dens, tf_pos=pos, tf_rgba=rgba, light_dir=base.light_dir,
                               light_radiance=base.light_radiance, env_radiance=base.env_radiance))
    return out
