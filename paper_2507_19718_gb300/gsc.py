"""Python binding of the GSCache CUDA library (``include/gsc.h``).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  If the library is
missing the first call raises (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

from . import build as _build

GSC_OK, GSC_ERR_INVALID_ARG, GSC_ERR_OOM, GSC_ERR_CUDA, GSC_ERR_CAPACITY, GSC_ERR_TIMEOUT, GSC_ERR_NOT_READY = range(7)
LOSS_HDR, LOSS_HDR_FULLGRAD, LOSS_L1_SSIM = 0, 1, 2
TR_OUT_CUMULATIVE, TR_OUT_PER_CALL = 0, 1
_STATUS_NAMES = ["OK", "INVALID_ARG", "OOM", "CUDA", "CAPACITY", "TIMEOUT", "NOT_READY"]


class GscError(RuntimeError):
    def __init__(self, status: int, message: str):
        name = _STATUS_NAMES[status] if 0 <= status < len(_STATUS_NAMES) else str(status)
        super().__init__(f"GSC_ERR_{name}: {message}")
        self.status = status


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("pos", C.c_float * 3), ("fx", C.c_float),
                ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32)]


class RasterCfg(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("list_capacity", C.c_int32),
                ("alpha_max", C.c_float), ("alpha_min", C.c_float), ("T_min", C.c_float),
                ("near_plane", C.c_float), ("dilation", C.c_float), ("bin_size", C.c_int32),
                ("pixels_per_thread", C.c_int32)]


class SceneDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("density", C.c_void_p),
                ("density_max", C.c_float), ("sigma_max", C.c_float), ("albedo", C.c_float),
                ("tf_count", C.c_int32), ("tf_pos", C.c_float * 16), ("tf_rgba", C.c_float * 64),
                ("light_dir", C.c_float * 3), ("light_radiance", C.c_float * 3), ("env_radiance", C.c_float * 3),
                ("n_spheres", C.c_int32), ("sphere_center", C.c_float * 12), ("sphere_radius", C.c_float * 4),
                ("sphere_radiance", C.c_float * 12)]


class TraceParams(C.Structure):
    _fields_ = [("spp", C.c_int32), ("max_bounces", C.c_int32), ("levels", C.c_int32), ("frame", C.c_uint32),
                ("seed", C.c_uint64), ("C", C.c_float), ("eps", C.c_float), ("tr_out", C.c_int32), ("pad", C.c_int32)]


class InitParams(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("levels", C.c_int32), ("max_attempts", C.c_int32), ("seed", C.c_uint64),
                ("opacity", C.c_float)]


class View(C.Structure):
    _fields_ = [("params", C.c_void_p), ("N", C.c_int64), ("cam", Camera), ("image", C.c_void_p),
                ("dL_dimage", C.c_void_p), ("grads", C.c_void_p)]


BATCH_FWD, BATCH_BWD = 1, 2


class TrainView(C.Structure):
    _fields_ = [("params", C.c_void_p), ("N", C.c_int64), ("cam", Camera), ("target", C.c_void_p),
                ("image", C.c_void_p), ("grads", C.c_void_p), ("loss", C.c_void_p)]


class Profile(C.Structure):
    _fields_ = [("n_phases", C.c_int32), ("names", (C.c_char * 16) * 24), ("ms", C.c_double * 24),
                ("launches", C.c_int64 * 24), ("calls", C.c_int64 * 24)]


class AdamParams(C.Structure):
    _fields_ = [("lr", C.c_float * 16), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("weight_decay", C.c_float), ("lr_scale", C.c_float), ("step", C.c_int32)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes); must cover every function of include/gsc.h
_vp, _i32, _i64, _f32, _sz = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_size_t
SIGNATURES = {
    "gsc_abi_version": (_i32, []),
    "gsc_last_error": (_i32, [C.c_char_p, _sz]),
    "gsc_scene_create": (_i32, [C.POINTER(SceneDesc), C.POINTER(_vp)]),
    "gsc_scene_set_tf": (_i32, [_vp, _i32, _vp, _vp]),
    "gsc_scene_destroy": (_i32, [_vp]),
    "gsc_trace": (_i32, [_vp, C.POINTER(Camera), C.POINTER(TraceParams), _vp, _vp, _vp, _vp]),
    "gsc_init_scratch_size": (_i32, [C.c_int64, C.POINTER(_sz)]),
    "gsc_cache_init": (_i32, [_vp, C.POINTER(InitParams), _vp, _sz, _vp, _vp]),
    "gsc_workspace_size": (_i32, [_i64, _i64, _i32, _i32, _i32, C.POINTER(RasterCfg), C.POINTER(_sz)]),
    "gsc_workspace_create": (_i32, [_vp, _sz, _i64, _i64, _i32, _i32, _i32, C.POINTER(RasterCfg),
                                    C.POINTER(_vp)]),
    "gsc_workspace_destroy": (_i32, [_vp]),
    "gsc_workspace_status": (_i32, [_vp, _vp, C.POINTER(_i64)]),
    "gsc_workspace_counters": (_i32, [_vp, _vp, C.POINTER(_i64), _i32]),
    "gsc_cache_render": (_i32, [_vp, _i64, C.POINTER(Camera), C.POINTER(RasterCfg), _vp, _vp, _vp]),
    "gsc_cache_backward": (_i32, [_vp, _i64, C.POINTER(Camera), C.POINTER(RasterCfg), _vp, _vp, _vp, _vp]),
    "gsc_render_batch": (_i32, [C.POINTER(View), _i32, _i32, C.POINTER(RasterCfg), _vp, _vp]),
    "gsc_train_batch": (_i32, [C.POINTER(TrainView), _i32, _i32, C.POINTER(RasterCfg), _vp, _vp]),
    "gsc_train_step": (_i32, [C.POINTER(TrainView), C.POINTER(_vp), C.POINTER(_vp), _i32, _i32,
                              C.POINTER(AdamParams), C.POINTER(RasterCfg), _vp, _vp]),
    "gsc_loss": (_i32, [_i32, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp]),
    "gsc_loss_noalloc": (_i32, [_i32, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp]),
    "gsc_cache_step": (_i32, [_vp, _vp, _vp, _vp, _i64, C.POINTER(AdamParams), _vp]),
    "gsc_lr_scale": (_f32, [_i32]),
    "gsc_profile_enable": (_i32, [_i32]),
    "gsc_profile_read": (_i32, [C.POINTER(Profile), _i32]),
    "gsc_launch_count": (_i64, []),
}


def library_path() -> str:
    return _build.SO


def lib(build_if_missing: bool = True):
    """The loaded CUDA library; builds it in-tree if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.SO
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"GSCache CUDA library missing at {path}; run build() first")
                _build.build()
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int):
    if status != GSC_OK:
        buf = C.create_string_buffer(512)
        lib().gsc_last_error(buf, 512)
        raise GscError(status, buf.value.decode(errors="replace"))


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _need(t: torch.Tensor, name: str, numel: int | None = None):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")


# ---------------------------------------------------------------- structs

def camera(cam) -> Camera:
    """gsc_camera from a ``synth.Camera``-like object (R, t, pos, fx, fy, cx, cy, width, height)."""
    c = Camera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).reshape(-1)]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float32)]
    c.pos[:] = [float(x) for x in np.asarray(cam.pos, np.float32)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def raster_cfg(tile=(16, 16), list_capacity: int = 256, alpha_max: float = 0.99, alpha_min: float = 1.0 / 255.0,
               T_min: float = 1e-4, near: float = 0.2, dilation: float = 0.3, bin_size: int = 0,
               pixels_per_thread: int = 1) -> RasterCfg:
    r = RasterCfg()
    r.pixels_per_thread = int(pixels_per_thread)
    r.tile_w, r.tile_h = int(tile[0]), int(tile[1])
    r.list_capacity = int(list_capacity)
    r.bin_size = int(bin_size)
    r.alpha_max, r.alpha_min, r.T_min, r.near_plane, r.dilation = alpha_max, alpha_min, T_min, near, dilation
    return r


def adam_params(lr, beta1=0.9, beta2=0.999, eps=1e-15, weight_decay=0.01, lr_scale=1.0, step=1) -> AdamParams:
    a = AdamParams()
    lr = list(np.asarray(lr, np.float32).reshape(-1))
    assert len(lr) == 16
    a.lr[:] = [float(x) for x in lr]
    a.beta1, a.beta2, a.eps, a.weight_decay, a.lr_scale, a.step = beta1, beta2, eps, weight_decay, lr_scale, int(step)
    return a


# Per-slot learning rates of the paper (Sec. 4.1): position 1.16e-3, opacity
# 1.5e-1, scaling 0, rotation 1e-3, colour 1.25e-2; pads 0.
PAPER_LR = np.array([1.16e-3, 1.16e-3, 1.16e-3, 1.5e-1, 0, 0, 0, 0, 1e-3, 1e-3, 1e-3, 1e-3, 1.25e-2, 1.25e-2,
                     1.25e-2, 0.0], np.float32)


# ---------------------------------------------------------------- scenes, tracer

class Scene:
    """A volume scene handle.  Keeps the caller's density tensor alive."""

    def __init__(self, density: torch.Tensor, density_max: float, sigma_max: float, albedo: float, tf_pos,
                 tf_rgba, light_dir, light_radiance, env_radiance, spheres=()):
        _need(density, "density")
        if density.dim() != 3:
            raise ValueError("density must be [nz, ny, nx]")
        self.density = density
        d = SceneDesc()
        d.nz, d.ny, d.nx = (int(s) for s in density.shape)
        d.density = density.data_ptr()
        d.density_max, d.sigma_max, d.albedo = density_max, sigma_max, albedo
        self._fill_tf(d, tf_pos, tf_rgba)
        d.light_dir[:] = [float(x) for x in light_dir]
        d.light_radiance[:] = [float(x) for x in light_radiance]
        d.env_radiance[:] = [float(x) for x in env_radiance]
        spheres = list(spheres or [])
        d.n_spheres = len(spheres)
        for l, (c, r, L) in enumerate(spheres[:4]):
            d.sphere_center[3 * l:3 * l + 3] = [float(x) for x in c]
            d.sphere_radius[l] = float(r)
            d.sphere_radiance[3 * l:3 * l + 3] = [float(x) for x in L]
        h = C.c_void_p()
        _check(lib().gsc_scene_create(C.byref(d), C.byref(h)))
        self.handle = h

    @staticmethod
    def _fill_tf(d, tf_pos, tf_rgba):
        pos = np.asarray(tf_pos, np.float32).reshape(-1)
        rgba = np.asarray(tf_rgba, np.float32).reshape(-1, 4)
        d.tf_count = len(pos)
        d.tf_pos[:len(pos)] = [float(x) for x in pos]
        d.tf_rgba[:rgba.size] = [float(x) for x in rgba.reshape(-1)]

    @classmethod
    def from_synth(cls, sc, device="cuda"):
        dens = torch.from_numpy(np.ascontiguousarray(sc.density)).to(device)
        return cls(dens, sc.density_max, sc.sigma_max, sc.albedo, sc.tf_pos, sc.tf_rgba, sc.light_dir,
                   sc.light_radiance, sc.env_radiance, getattr(sc, "spheres", ()))

    def set_tf(self, tf_pos, tf_rgba):
        pos = np.ascontiguousarray(np.asarray(tf_pos, np.float32).reshape(-1))
        rgba = np.ascontiguousarray(np.asarray(tf_rgba, np.float32).reshape(-1, 4))
        _check(lib().gsc_scene_set_tf(self.handle, len(pos), pos.ctypes.data_as(C.c_void_p),
                                      rgba.ctypes.data_as(C.c_void_p)))

    def close(self):
        if getattr(self, "handle", None):
            lib().gsc_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace(scene: Scene, cam, spp: int, max_bounces: int, levels: int, seed: int, frame: int = 0, C_term: float = 0.0,
          eps: float = 1e-6, cache: torch.Tensor | None = None, targets: torch.Tensor | None = None,
          image: torch.Tensor | None = None, stream=None, tr_out: int = 0):
    """gsc_trace: returns (targets [K,3,H,W], image [3,H,W]).  tr_out: reading
    of Algorithm 1's Tr_out (TR_OUT_CUMULATIVE or TR_OUT_PER_CALL)."""
    c = cam if isinstance(cam, Camera) else camera(cam)
    H, W = c.height, c.width
    dev = scene.density.device
    if image is None:
        image = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    if targets is None and levels > 0:
        targets = torch.empty((levels, 3, H, W), dtype=torch.float32, device=dev)
    _need(image, "image", 3 * H * W)
    if levels > 0:
        _need(targets, "targets", levels * 3 * H * W)
    if cache is not None:
        _need(cache, "cache", levels * 3 * H * W)
    p = TraceParams()
    p.spp, p.max_bounces, p.levels, p.frame, p.seed, p.C, p.eps = spp, max_bounces, levels, frame, seed, C_term, eps
    p.tr_out = int(tr_out)
    _check(lib().gsc_trace(scene.handle, C.byref(c), C.byref(p), _ptr(cache), _ptr(targets), _ptr(image),
                           _stream(stream)))
    return targets, image


def cache_init(scene: Scene, n_points: int, levels: int, seed: int, opacity: float = 0.1, max_attempts: int = 0,
               stream=None):
    """gsc_cache_init: the initial cache of Sec. 3.2 / Eq. 3.  Returns the
    (sum_k N >> k, 16) parameter tensor and its per-level views."""
    dev = scene.density.device
    nbytes = _sz()
    _check(lib().gsc_init_scratch_size(n_points, C.byref(nbytes)))
    scratch = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=dev)
    base = (scratch.data_ptr() + 255) & ~255
    sizes = [n_points >> k for k in range(levels)]
    params = torch.empty((sum(sizes), 16), dtype=torch.float32, device=dev)
    p = InitParams()
    p.n_points, p.levels, p.max_attempts, p.seed, p.opacity = n_points, levels, max_attempts, seed, opacity
    _check(lib().gsc_cache_init(scene.handle, C.byref(p), C.c_void_p(base), nbytes.value, params.data_ptr(),
                                _stream(stream)))
    out, r = [], 0
    for n in sizes:
        out.append(params[r:r + n])
        r += n
    return params, out


# ---------------------------------------------------------------- workspaces, raster

class Workspace:
    """Rasterizer workspace in a torch-allocated device buffer."""

    def __init__(self, max_gaussians: int, max_pairs: int, max_w: int, max_h: int, device="cuda",
                 max_views: int = 1):
        nbytes = C.c_size_t()
        _check(lib().gsc_workspace_size(max_gaussians, max_pairs, max_w, max_h, max_views, None,
                                        C.byref(nbytes)))
        self.nbytes = nbytes.value
        self.buffer = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        base = self.buffer.data_ptr()
        aligned = (base + 255) & ~255
        h = C.c_void_p()
        _check(lib().gsc_workspace_create(C.c_void_p(aligned), self.nbytes, max_gaussians, max_pairs, max_w, max_h,
                                          max_views, None, C.byref(h)))
        self.handle = h
        self.max_gaussians, self.max_pairs, self.max_w, self.max_h = max_gaussians, max_pairs, max_w, max_h

    def status(self, stream=None) -> int:
        """Synchronise; raise GscError on a device-side error; return the
        largest pair count requested since the last call."""
        need = C.c_int64()
        _check(lib().gsc_workspace_status(self.handle, _stream(stream), C.byref(need)))
        return need.value

    def counters(self, stream=None) -> dict:
        """Synchronise and return (then reset) the workspace's work counters."""
        out = (C.c_int64 * 12)()
        _check(lib().gsc_workspace_counters(self.handle, _stream(stream), out, 12))
        return dict(pairs_last=out[0], pairs_max=out[1], eval_fwd=out[2], composited_fwd=out[3],
                    eval_rewalk=out[4], eval_back=out[5], pairs_sum=out[6], binnings=out[7],
                    composited_rewalk=out[8], hits_back=out[9], items_last=out[10], pairs_culled=out[11])

    def close(self):
        if getattr(self, "handle", None):
            lib().gsc_workspace_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cache_render(params: torch.Tensor, cam, cfg: RasterCfg, ws: Workspace, image: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    c = cam if isinstance(cam, Camera) else camera(cam)
    _need(params, "params")
    N = params.numel() // 16
    if image is None:
        image = torch.empty((3, c.height, c.width), dtype=torch.float32, device=params.device)
    _need(image, "image", 3 * c.height * c.width)
    _check(lib().gsc_cache_render(_ptr(params), N, C.byref(c), C.byref(cfg), ws.handle, _ptr(image),
                                  _stream(stream)))
    return image


def cache_backward(params: torch.Tensor, cam, cfg: RasterCfg, ws: Workspace, dL_dimage: torch.Tensor,
                   grads: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    c = cam if isinstance(cam, Camera) else camera(cam)
    _need(params, "params")
    _need(dL_dimage, "dL_dimage", 3 * c.height * c.width)
    N = params.numel() // 16
    if grads is None:
        grads = torch.zeros_like(params)
    _need(grads, "grads", params.numel())
    _check(lib().gsc_cache_backward(_ptr(params), N, C.byref(c), C.byref(cfg), ws.handle, _ptr(dL_dimage),
                                    _ptr(grads), _stream(stream)))
    return grads


def render_batch(views, mode: int, cfg: RasterCfg, ws: Workspace, stream=None):
    """gsc_render_batch.  views: sequence of dicts with params (N x 16), cam,
    and image (forward) / dL_dimage + grads (backward) tensors."""
    arr = (View * len(views))()
    for i, v in enumerate(views):
        p = v["params"]
        _need(p, "params")
        c = v["cam"] if isinstance(v["cam"], Camera) else camera(v["cam"])
        arr[i].params = p.data_ptr()
        arr[i].N = p.numel() // 16
        arr[i].cam = c
        npx = 3 * c.width * c.height
        if mode & BATCH_FWD:
            _need(v["image"], "image", npx)
            arr[i].image = v["image"].data_ptr()
        if mode & BATCH_BWD:
            _need(v["dL_dimage"], "dL_dimage", npx)
            _need(v["grads"], "grads", p.numel())
            arr[i].dL_dimage = v["dL_dimage"].data_ptr()
            arr[i].grads = v["grads"].data_ptr()
    _check(lib().gsc_render_batch(arr, len(views), mode, C.byref(cfg), ws.handle, _stream(stream)))


def _train_views(views):
    arr = (TrainView * len(views))()
    for i, v in enumerate(views):
        p = v["params"]
        _need(p, "params")
        c = v["cam"] if isinstance(v["cam"], Camera) else camera(v["cam"])
        npx = 3 * c.width * c.height
        _need(v["target"], "target", npx)
        arr[i].params = p.data_ptr()
        arr[i].N = p.numel() // 16
        arr[i].cam = c
        arr[i].target = v["target"].data_ptr()
        if v.get("grads") is not None:  # train_step: optional (no accumulated gradient)
            _need(v["grads"], "grads", p.numel())
            arr[i].grads = v["grads"].data_ptr()
        _need(v["loss"], "loss", 1)
        arr[i].loss = v["loss"].data_ptr()
        if v.get("image") is not None:
            _need(v["image"], "image", npx)
            arr[i].image = v["image"].data_ptr()
    return arr


def train_batch(views, cfg: RasterCfg, ws: Workspace, loss_kind: int = 0, stream=None):
    """gsc_train_batch: render + HDR loss + backward of every view in one
    launch.  views: dicts with params (N x 16), cam, target (3 x H x W),
    grads (N x 16, +=), loss (device scalar) and optionally image."""
    arr = _train_views(views)
    _check(lib().gsc_train_batch(arr, len(views), loss_kind, C.byref(cfg), ws.handle, _stream(stream)))


def train_step(views, adam: AdamParams, cfg: RasterCfg, ws: Workspace, loss_kind: int = 0, stream=None):
    """gsc_train_step: train_batch with the AdamW step of every view's
    parameters fused into the gradient kernel.  views: as train_batch plus m
    and v (N x 16 each); params are updated in place; grads (optional) is an
    accumulated gradient, read and zeroed; views must not share parameters."""
    arr = _train_views(views)
    M = (_vp * len(views))()
    V = (_vp * len(views))()
    for i, v in enumerate(views):
        n = v["params"].numel()
        _need(v["m"], "m", n)
        _need(v["v"], "v", n)
        M[i] = v["m"].data_ptr()
        V[i] = v["v"].data_ptr()
    _check(lib().gsc_train_step(arr, M, V, len(views), loss_kind, C.byref(adam), C.byref(cfg), ws.handle,
                                _stream(stream)))


def loss(kind: int, pred: torch.Tensor, target: torch.Tensor, ws: Workspace, crop=None,
         dL_dpred: torch.Tensor | None = None, loss_out: torch.Tensor | None = None, want_grad: bool = True,
         stream=None):
    _need(pred, "pred")
    _need(target, "target", pred.numel())
    Cc, H, W = pred.shape
    if want_grad and dL_dpred is None:
        dL_dpred = torch.empty_like(pred)
    if loss_out is None:
        loss_out = torch.empty((), dtype=torch.float32, device=pred.device)
    cr = None
    if crop is not None:
        cr = (C.c_int32 * 4)(*[int(x) for x in crop])
    _check(lib().gsc_loss(kind, _ptr(pred), _ptr(target), Cc, H, W, cr, _ptr(dL_dpred) if want_grad else None,
                          _ptr(loss_out), ws.handle, _stream(stream)))
    return loss_out, dL_dpred


def loss_noalloc(kind: int, pred: torch.Tensor, target: torch.Tensor, crop=None,
                 dL_dpred: torch.Tensor | None = None, loss_out: torch.Tensor | None = None,
                 want_grad: bool = True, stream=None):
    """gsc_loss_noalloc: the loss without a workspace (the library's own
    fixed scratch; at most 8,388,608 elements)."""
    _need(pred, "pred")
    _need(target, "target", pred.numel())
    Cc, H, W = pred.shape
    if want_grad and dL_dpred is None:
        dL_dpred = torch.empty_like(pred)
    if loss_out is None:
        loss_out = torch.empty((), dtype=torch.float32, device=pred.device)
    cr = (C.c_int32 * 4)(*[int(x) for x in crop]) if crop is not None else None
    _check(lib().gsc_loss_noalloc(kind, _ptr(pred), _ptr(target), Cc, H, W, cr,
                                  _ptr(dL_dpred) if want_grad else None, _ptr(loss_out), _stream(stream)))
    return loss_out, dL_dpred


def cache_step(params, grads, m, v, adam: AdamParams, stream=None):
    for t, n in ((params, "params"), (grads, "grads"), (m, "m"), (v, "v")):
        _need(t, n, params.numel())
    _check(lib().gsc_cache_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), params.numel() // 16, C.byref(adam),
                                _stream(stream)))


def lr_scale(t: int) -> float:
    return lib().gsc_lr_scale(int(t))


# ---------------------------------------------------------------- instrumentation

def profile_enable(on: bool = True):
    _check(lib().gsc_profile_enable(1 if on else 0))


def profile_read(reset: bool = True) -> dict:
    """{phase: (ms, launches, calls)} of the event-timed kernel phases."""
    p = Profile()
    _check(lib().gsc_profile_read(C.byref(p), 1 if reset else 0))
    return {p.names[k].value.decode(): (p.ms[k], p.launches[k], p.calls[k]) for k in range(p.n_phases)}


def launch_count() -> int:
    return lib().gsc_launch_count()


# ---------------------------------------------------------------- autograd

class CacheRender(torch.autograd.Function):
    """Differentiable render of one cache level.  Saves only the parameters;
    the backward re-bins and re-sorts (gsc_cache_backward keeps no per-pixel
    forward state)."""

    @staticmethod
    def forward(ctx, params, cam, cfg, ws):
        ctx.save_for_backward(params)
        ctx.cam, ctx.cfg, ctx.ws = cam, cfg, ws
        return cache_render(params.contiguous(), cam, cfg, ws)

    @staticmethod
    def backward(ctx, dimg):
        (params,) = ctx.saved_tensors
        grads = torch.zeros_like(params)
        cache_backward(params.contiguous(), ctx.cam, ctx.cfg, ctx.ws, dimg.contiguous(), grads)
        return grads, None, None, None


def render(params, cam, cfg, ws):
    return CacheRender.apply(params, cam if isinstance(cam, Camera) else camera(cam), cfg, ws)
