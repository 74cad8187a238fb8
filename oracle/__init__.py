"""CPU oracle of the GSCache hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct restatement of what the CUDA path computes,
in FP64 C (``gsc_oracle.c``, ``trace_body.inc``) with this thin ctypes
wrapper.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import it.  The product path never does:
it shares no code with the CUDA library, and the CUDA library never falls back
to it.

Passages followed (Bauer et al., "GSCache"):
  trace              Sec. 3.1 Eq. 1, Sec. 3.2, Sec. 3.3 + Algorithm 1,
                     Sec. 3.4 Eq. 2, Sec. 3.5 (intermediate path buffers)
  project / render   Sec. 3.1 (Gaussian splatting of each cache level)
  render_backward    Sec. 3.5 ("inverse splatting step"); render_backward_terms,
                     project_backward and grad_abs_map for the rounding bounds
                     of an FP32 implementation
  render_leaves,     the same with every decision within 2e-4 of its
  render_backward_bounds  threshold taken both ways
  init_*             Sec. 3.2 "Cache Initialization" and Eq. 3
  FrozenLists        the same render with its threshold decisions held fixed,
                     for central differences of the backward at 1M Gaussians
  loss_hdr           Sec. 3.6 "Loss"
  adamw              Sec. 3.6 "Regularization"; lr_scale Eq. 4
  cache_bytes        Table 3
  loss_l1ssim        not in the paper (the 1M-Gaussian gradient workload)

The cache-coupled tracer branch (Algorithm 1 with C > 0 and cache images) is
pinned by the C -> infinity identity and by three closed forms in a
homogeneous medium with constant cache images: C -> 0+ (every collision ends
in the first cache level), one survival with weight 1/Tr followed by an escape
into the cache from a dense half-space (escape probability (1 - ln 2) / 2),
and no roulette from Tr = 0.9 up.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRCS = [os.path.join(_HERE, "gsc_oracle.c"), os.path.join(_HERE, "trace_body.inc")]
_lock = threading.Lock()
_lib = None

RASTER_DEFAULTS = dict(alpha_max=0.99, alpha_min=1.0 / 255.0, T_min=1e-4, near=0.2, dilation=0.3)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRCS[0], "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            vp, i32, i64, f32, f64, u32, u64 = C.c_void_p, C.c_int, C.c_int64, C.c_float, C.c_double, C.c_uint32, C.c_uint64
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_ln_f32.argtypes = [vp, vp, i64]
            L.orc_sincos2pi_f32.argtypes = [vp, vp, vp, i64]
            L.orc_trace.argtypes = [i32, vp, i32, i32, i32, vp, i32, vp, vp, vp, i32, vp, vp, i32, i32, i32, i32, i32,
                                    u64, u32, f32, f32, i32, vp, i32, i32, i32, i32, vp, vp, vp, i32]
            L.orc_trace.restype = i32
            L.orc_transmittance.argtypes = [i32, vp, i32, i32, i32, vp, i32, vp, vp, vp, vp, i64, u64, vp, i32]
            L.orc_sigma_t.argtypes = [vp, i32, i32, i32, vp, i32, vp, vp, vp, i64, vp]
            L.orc_project.argtypes = [i64, vp, vp, vp, vp]
            L.orc_render.argtypes = [i64, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, vp, i32, i32]
            L.orc_render.restype = i32
            L.orc_render_backward.argtypes = [i64, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, i32]
            L.orc_render_backward.restype = i32
            L.orc_render_backward_ex.argtypes = [i64, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, vp, vp, i32]
            L.orc_render_backward_ex.restype = i32
            L.orc_grad_abs_map.argtypes = [i64, vp, vp, vp, vp, vp, i32]
            L.orc_render_leaves.argtypes = [i64, vp, vp, vp, i32, i32, i32, i32, i32, vp, vp, i32]
            L.orc_render_leaves.restype = i32
            L.orc_render_backward_bounds.argtypes = [i64, vp, vp, vp, i32, i32, i32, i32, vp, i32, vp, vp, vp, vp,
                                                     vp, i32]
            L.orc_render_backward_bounds.restype = i32
            L.orc_project_backward.argtypes = [i64, vp, vp, vp, vp, vp, i32]
            L.orc_render_lists.argtypes = [i64, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, i32]
            L.orc_render_lists.restype = i32
            L.orc_frozen_fd.argtypes = [i64, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, vp, i32, vp, vp, f64, vp,
                                        i32]
            L.orc_frozen_fd.restype = i32
            L.orc_render_frozen.argtypes = [i64, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, vp, i32]
            L.orc_render_frozen.restype = i32
            L.orc_init_points.argtypes = [i32, vp, i32, i32, i32, vp, i32, vp, vp, i64, vp, u64, i32, vp, vp, vp,
                                          i32]
            L.orc_knn3_mean.argtypes = [vp, i64, vp, i64, vp, i32]
            L.orc_init_scales.argtypes = [vp, i64, vp, vp, vp]
            L.orc_loss_hdr.argtypes = [vp, vp, i32, i32, i32, vp, i32, vp]
            L.orc_loss_hdr.restype = f64
            L.orc_loss_l1ssim.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp]
            L.orc_loss_l1ssim.restype = f64
            L.orc_adamw.argtypes = [i64, vp, vp, vp, vp, vp, f64, f64, f64, f64, f64, i32]
            L.orc_lr_scale.argtypes = [i32]
            L.orc_lr_scale.restype = f64
            L.orc_cache_bytes.argtypes = [i64]
            L.orc_cache_bytes.restype = i64
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype))


def _threads(n):
    return int(n) if n else (os.cpu_count() or 1)


# ---------------------------------------------------------------- RNG / math

def philox4x32_10(ctr, key) -> np.ndarray:
    c, k, out = _c(ctr, np.uint32), _c(key, np.uint32), np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def ln_f32(x) -> np.ndarray:
    x = _c(x, np.float32)
    y = np.empty_like(x)
    lib().orc_ln_f32(_p(x), _p(y), x.size)
    return y


def sincos2pi_f32(u):
    u = _c(u, np.float32)
    s, c = np.empty_like(u), np.empty_like(u)
    lib().orc_sincos2pi_f32(_p(u), _p(s), _p(c), u.size)
    return s, c


# ---------------------------------------------------------------- tracer

def _scene_arrays(scene):
    grid = _c(scene.density, np.float32)
    nz, ny, nx = grid.shape
    vol_f = np.array([scene.density_max, scene.sigma_max, scene.albedo], np.float32)
    tf_pos = _c(scene.tf_pos, np.float32)
    tf_rgba = _c(scene.tf_rgba, np.float32)
    light = np.concatenate([scene.light_dir, scene.light_radiance, scene.env_radiance]).astype(np.float32)
    sph = getattr(scene, "spheres", None) or []
    spheres = np.array([[*c, r, *L] for c, r, L in sph], np.float32).reshape(-1, 7)
    return grid, nx, ny, nz, vol_f, tf_pos, tf_rgba, (light, spheres)


def trace(scene, cam, spp: int, max_bounces: int, levels: int, seed: int, frame: int = 0, C: float = 0.0,
          eps: float = 1e-6, cache=None, window=None, precision: int = 64, nthreads: int = 0,
          lengths: bool = False, tr_out: int = 0):
    """Image (3, h, w) and K target buffers (K, 3, h, w) over ``window``
    (x0, y0, w, h; default the whole frame).  precision 32 = FP32 mirror.
    tr_out: reading of Algorithm 1's Tr_out, 0 cumulative, 1 per call."""
    grid, nx, ny, nz, vol_f, tf_pos, tf_rgba, (light, spheres) = _scene_arrays(scene)
    W, H = cam.width, cam.height
    x0, y0, w, h = window if window is not None else (0, 0, W, H)
    camp = cam.packed()
    targets = np.zeros((levels, 3, h, w), np.float64)
    image = np.zeros((3, h, w), np.float64)
    lens = np.zeros((h, w, spp), np.int32) if lengths else None
    cache_a = _c(cache, np.float32) if cache is not None else None
    rc = lib().orc_trace(precision, _p(grid), nx, ny, nz, _p(vol_f), len(tf_pos), _p(tf_pos), _p(tf_rgba),
                         _p(light), len(spheres), _p(spheres), _p(camp), W, H, spp, max_bounces, levels, seed, frame, C, eps,
                         int(tr_out), _p(cache_a),
                         x0, y0, w, h, _p(targets), _p(image), _p(lens), _threads(nthreads))
    if rc != 0:
        raise ValueError(f"orc_trace rejected its arguments (code {rc})")
    return (targets, image, lens) if lengths else (targets, image)


def transmittance(mode: str, scene, origin, direction, n: int, seed: int, nthreads: int = 0) -> np.ndarray:
    grid, nx, ny, nz, vol_f, tf_pos, tf_rgba, _ = _scene_arrays(scene)
    o, d = _c(origin, np.float64), _c(direction, np.float64)
    out = np.empty(n, np.float64)
    lib().orc_transmittance({"delta": 0, "ratio": 1}[mode], _p(grid), nx, ny, nz, _p(vol_f), len(tf_pos),
                            _p(tf_pos), _p(tf_rgba), _p(o), _p(d), n, seed, _p(out), _threads(nthreads))
    return out


def sigma_t(scene, pts) -> np.ndarray:
    grid, nx, ny, nz, vol_f, tf_pos, tf_rgba, _ = _scene_arrays(scene)
    pts = _c(pts, np.float64).reshape(-1, 3)
    out = np.empty(len(pts), np.float64)
    lib().orc_sigma_t(_p(grid), nx, ny, nz, _p(vol_f), len(tf_pos), _p(tf_pos), _p(tf_rgba), _p(pts), len(pts),
                      _p(out))
    return out


# ---------------------------------------------------------------- cache initialisation

INIT_MAX_ATTEMPTS = 4096


def init_points(scene, n: int, seed: int, idx=None, precision: int = 32, max_attempts: int = INIT_MAX_ATTEMPTS,
                nthreads: int = 0):
    """Delta-tracked point samples (Sec. 3.2): positions (n, 3), albedos (n, 3),
    attempts (n,) for points 0..n-1 or the given indices."""
    grid, nx, ny, nz, vol_f, tf_pos, tf_rgba, _ = _scene_arrays(scene)
    ix = _c(idx, np.int64) if idx is not None else None
    m = len(ix) if ix is not None else n
    pos = np.zeros((m, 3), np.float64)
    alb = np.zeros((m, 3), np.float64)
    att = np.zeros(m, np.int32)
    lib().orc_init_points(precision, _p(grid), nx, ny, nz, _p(vol_f), len(tf_pos), _p(tf_pos), _p(tf_rgba), m,
                          _p(ix), seed, max_attempts, _p(pos), _p(alb), _p(att), _threads(nthreads))
    return pos, alb, att


def knn3_mean(pts, query=None, nthreads: int = 0) -> np.ndarray:
    """Mean distance of each (query) point to its three nearest others, brute force."""
    pts = _c(pts, np.float64).reshape(-1, 3)
    q = _c(query, np.int64) if query is not None else None
    out = np.zeros(len(q) if q is not None else len(pts), np.float64)
    lib().orc_knn3_mean(_p(pts), len(pts), _p(q), len(out), _p(out), _threads(nthreads))
    return out


def init_scales(mbar):
    """Eq. 3: isotropic scales from the mean 3-NN distances; returns (s, mu, sigma)."""
    mbar = _c(mbar, np.float64)
    s = np.zeros_like(mbar)
    mu, sg = C.c_double(), C.c_double()
    lib().orc_init_scales(_p(mbar), len(mbar), _p(s), C.byref(mu), C.byref(sg))
    return s, mu.value, sg.value


def init_gaussians(scene, n_points: int, levels: int, seed: int, opacity: float = 0.1, precision: int = 32,
                   nthreads: int = 0):
    """The initial cache: level k holds points 0 .. (n_points >> k) - 1 of one
    sampled cloud, each a Gaussian at the point with the point's albedo as
    colour, identity rotation, the given opacity and the Eq. 3 scale from the
    3-NN distances within its level.  Returns one (N_k, 16) array per level."""
    pos, alb, att = init_points(scene, n_points, seed, precision=precision, nthreads=nthreads)
    if (att == 0).any():
        raise RuntimeError("some points found no interaction")
    pos32 = pos.astype(np.float32).astype(np.float64)
    out = []
    for k in range(levels):
        n = n_points >> k
        mbar = knn3_mean(pos32[:n], nthreads=nthreads)
        s, _, _ = init_scales(mbar)
        p = np.zeros((n, 16), np.float64)
        p[:, 0:3] = pos32[:n]
        p[:, 3] = np.log(opacity / (1.0 - opacity))
        p[:, 4:7] = np.log(s)[:, None]
        p[:, 8] = 1.0
        p[:, 12:15] = alb[:n]
        out.append(p)
    return out


# ---------------------------------------------------------------- rasterizer

def _cfg(cfg):
    d = dict(RASTER_DEFAULTS)
    if cfg:
        d.update(cfg)
    return np.array([d["alpha_max"], d["alpha_min"], d["T_min"], d["near"], d["dilation"]], np.float64)


def project(params, cam, cfg=None) -> np.ndarray:
    """(N, 11): mx, my, a, b, c, opacity, r, g, b, depth(FP32), visible."""
    params = _c(params, np.float32)
    out = np.zeros((len(params), 11), np.float64)
    lib().orc_project(len(params), _p(params), _p(cam.packed()), _p(_cfg(cfg)), _p(out))
    return out


def render(params, cam, cfg=None, window=None, nthreads: int = 0, grad_margins: bool = False):
    """Returns image (3, h, w), marginal (h, w) bool, ncontrib (h, w), T_final (h, w).

    marginal flags pixels where a compositing decision lay within 2e-4
    (relative) of its threshold, so that an FP32 implementation may take it
    the other way; grad_margins also flags terms near the alpha_max clamp."""
    params = _c(params, np.float32)
    x0, y0, w, h = window if window is not None else (0, 0, cam.width, cam.height)
    image = np.zeros((3, h, w), np.float64)
    marg = np.zeros((h, w), np.uint8)
    ncon = np.zeros((h, w), np.int32)
    tfin = np.zeros((h, w), np.float64)
    rc = lib().orc_render(len(params), _p(params), _p(cam.packed()), _p(_cfg(cfg)), x0, y0, w, h, _p(image),
                          _p(marg), _p(ncon), _p(tfin), int(grad_margins), _threads(nthreads))
    if rc:
        raise MemoryError("orc_render")
    return image, marg.astype(bool), ncon, tfin


def render_backward(params, cam, dL_dimage, cfg=None, window=None, nthreads: int = 0):
    """Returns grads (N, 16) and 2D grads (N, 9) of sum(dL_dimage * render)."""
    params = _c(params, np.float32)
    x0, y0, w, h = window if window is not None else (0, 0, cam.width, cam.height)
    g = _c(dL_dimage, np.float64)
    assert g.shape == (3, h, w)
    grads = np.zeros((len(params), 16), np.float64)
    g2d = np.zeros((len(params), 9), np.float64)
    rc = lib().orc_render_backward(len(params), _p(params), _p(cam.packed()), _p(_cfg(cfg)), x0, y0, w, h, _p(g),
                                   _p(grads), _p(g2d), _threads(nthreads))
    if rc:
        raise MemoryError("orc_render_backward")
    return grads, g2d


def render_backward_terms(params, cam, dL_dimage, cfg=None, window=None, nthreads: int = 0):
    """render_backward plus, per Gaussian, the sum of the absolute values of
    the (pixel, term) contributions to each 2D gradient component (N, 9) and
    the number of contributions (N,): the conditioning of each gradient sum,
    which bounds the rounding error of a low-precision implementation."""
    params = _c(params, np.float32)
    x0, y0, w, h = window if window is not None else (0, 0, cam.width, cam.height)
    g = _c(dL_dimage, np.float64)
    assert g.shape == (3, h, w)
    grads = np.zeros((len(params), 16), np.float64)
    g2d = np.zeros((len(params), 9), np.float64)
    a2d = np.zeros((len(params), 9), np.float64)
    nterm = np.zeros(len(params), np.int64)
    rc = lib().orc_render_backward_ex(len(params), _p(params), _p(cam.packed()), _p(_cfg(cfg)), x0, y0, w, h,
                                      _p(g), _p(grads), _p(g2d), _p(a2d), _p(nterm), _threads(nthreads))
    if rc:
        raise MemoryError("orc_render_backward_ex")
    return grads, g2d, a2d, nterm


def grad_abs_map(params, cam, abs2d, cfg=None, nthreads: int = 0) -> np.ndarray:
    """Magnitude of the packed parameter gradient (N, 16) for 2D records of
    magnitude abs2d (N, 9): the projection backward evaluated on absolute
    values (it bounds |J a| for |a| <= abs2d, J the Jacobian, and the
    intermediate values of the computation)."""
    params = _c(params, np.float32)
    m = _c(abs2d, np.float64)
    assert m.shape == (len(params), 9)
    out = np.zeros((len(params), 16), np.float64)
    lib().orc_grad_abs_map(len(params), _p(params), _p(cam.packed()), _p(_cfg(cfg)), _p(m), _p(out),
                           _threads(nthreads))
    return out


def render_leaves(params, cam, cfg=None, window=None, max_leaves: int = 64, nthreads: int = 0):
    """Every value a pixel may take when its marginal compositing decisions
    (alpha_min and T_min within the margin) go either way: leaves
    (h, w, max_leaves, 3) and their count (h, w); -1 marks a pixel with more
    than max_leaves.  One leaf where nothing is marginal: render's value."""
    params = _c(params, np.float32)
    x0, y0, w, h = window if window is not None else (0, 0, cam.width, cam.height)
    leaves = np.zeros((h, w, max_leaves, 3), np.float64)
    n = np.zeros((h, w), np.int32)
    rc = lib().orc_render_leaves(len(params), _p(params), _p(cam.packed()), _p(_cfg(cfg)), x0, y0, w, h, max_leaves,
                                 _p(leaves), _p(n), _threads(nthreads))
    if rc:
        raise MemoryError("orc_render_leaves")
    return leaves, n


def render_backward_bounds(params, cam, dL_dimage, cfg=None, window=None, max_leaves: int = 64, nthreads: int = 0):
    """Bounds of the 2D gradient record over every way the marginal
    decisions (alpha_min, T_min, alpha_max clamp) may go: lo2d, hi2d (N, 9),
    the per-pixel largest absolute contributions summed (N, 9), the number of
    contributing pixels (N,) and the leaves per pixel (h, w; -1 beyond
    max_leaves)."""
    params = _c(params, np.float32)
    x0, y0, w, h = window if window is not None else (0, 0, cam.width, cam.height)
    g = _c(dL_dimage, np.float64)
    assert g.shape == (3, h, w)
    n = len(params)
    lo, hi, ab = (np.zeros((n, 9), np.float64) for _ in range(3))
    nterm = np.zeros(n, np.int64)
    nl = np.zeros((h, w), np.int32)
    rc = lib().orc_render_backward_bounds(n, _p(params), _p(cam.packed()), _p(_cfg(cfg)), x0, y0, w, h, _p(g),
                                          max_leaves, _p(lo), _p(hi), _p(ab), _p(nterm), _p(nl), _threads(nthreads))
    if rc:
        raise MemoryError("orc_render_backward_bounds")
    return lo, hi, ab, nterm, nl


def project_backward(params, cam, g2d, cfg=None, nthreads: int = 0) -> np.ndarray:
    """The packed parameter gradient (N, 16) of 2D gradient records (N, 9)."""
    params = _c(params, np.float32)
    a = _c(g2d, np.float64)
    assert a.shape == (len(params), 9)
    out = np.zeros((len(params), 16), np.float64)
    lib().orc_project_backward(len(params), _p(params), _p(cam.packed()), _p(_cfg(cfg)), _p(a), _p(out),
                               _threads(nthreads))
    return out


class FrozenLists:
    """Per-pixel composited lists of a window (Gaussian ids in compositing
    order and their alpha_max clamp state), recorded at given parameters."""

    def __init__(self, params, cam, cfg=None, window=None, nthreads: int = 0):
        params = _c(params, np.float32)
        self.window = tuple(window) if window is not None else (0, 0, cam.width, cam.height)
        x0, y0, w, h = self.window
        _, _, ncon, _ = render(params, cam, cfg, self.window, nthreads, grad_margins=True)
        self.offsets = np.zeros(w * h + 1, np.int64)
        np.cumsum(ncon.reshape(-1), out=self.offsets[1:])
        n = int(self.offsets[-1])
        self.g = np.zeros(max(n, 1), np.int64)
        self.clamped = np.zeros(max(n, 1), np.uint8)
        rc = lib().orc_render_lists(len(params), _p(params), _p(cam.packed()), _p(_cfg(cfg)), x0, y0, w, h,
                                    _p(self.offsets), _p(self.g), _p(self.clamped), _threads(nthreads))
        if rc:
            raise RuntimeError(f"orc_render_lists: {rc}")
        self.cam, self.cfg = cam, cfg

    def render(self, params, nthreads: int = 0) -> np.ndarray:
        """The window rendered over the frozen lists (3, h, w)."""
        params = _c(params, np.float32)
        x0, y0, w, h = self.window
        img = np.zeros((3, h, w), np.float64)
        rc = lib().orc_render_frozen(len(params), _p(params), _p(self.cam.packed()), _p(_cfg(self.cfg)), x0, y0, w,
                                     h, _p(self.offsets), _p(self.g), _p(self.clamped), _p(img), _threads(nthreads))
        if rc:
            raise MemoryError("orc_render_frozen")
        return img

    def fd(self, params, v, gauss, slots, h: float = 1e-3, nthreads: int = 0) -> np.ndarray:
        """Central differences of sum(v * frozen render) w.r.t. params[gauss[i], slots[i]]."""
        params = _c(params, np.float32)
        x0, y0, w, hh = self.window
        v = _c(v, np.float64)
        assert v.shape == (3, hh, w)
        gauss, slots = _c(gauss, np.int64), _c(slots, np.int32)
        out = np.zeros(len(gauss), np.float64)
        rc = lib().orc_frozen_fd(len(params), _p(params), _p(self.cam.packed()), _p(_cfg(self.cfg)), x0, y0, w, hh,
                                 _p(self.offsets), _p(self.g), _p(self.clamped), _p(v), len(gauss), _p(gauss),
                                 _p(slots), float(h), _p(out), _threads(nthreads))
        if rc:
            raise MemoryError("orc_frozen_fd")
        return out


# ---------------------------------------------------------------- losses, optimiser

def loss_hdr(pred, target, crop=None, full_grad: bool = False):
    pred, target = _c(pred, np.float32), _c(target, np.float32)
    Cc, H, W = pred.shape
    grad = np.zeros((Cc, H, W), np.float64)
    cr = _c(crop, np.int32) if crop is not None else None
    val = lib().orc_loss_hdr(_p(pred), _p(target), Cc, H, W, _p(cr), int(full_grad), _p(grad))
    return val, grad


def loss_l1ssim(pred, target, crop=None):
    pred, target = _c(pred, np.float32), _c(target, np.float32)
    Cc, H, W = pred.shape
    grad = np.zeros((Cc, H, W), np.float64)
    cr = _c(crop, np.int32) if crop is not None else None
    w, h = (crop[2], crop[3]) if crop is not None else (W, H)
    smap = np.zeros((Cc, h, w), np.float64)
    val = lib().orc_loss_l1ssim(_p(pred), _p(target), Cc, H, W, _p(cr), _p(grad), _p(smap))
    return val, grad, smap


def adamw(p, g, m, v, lr, lr_scale=1.0, beta1=0.9, beta2=0.999, eps=1e-15, weight_decay=0.01, step=1):
    """In-place FP64 AdamW step on flat (N*16) arrays; zeroes g."""
    arrs = [p, g, m, v]
    for a in arrs:
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lr = _c(lr, np.float64)
    assert lr.size == 16
    lib().orc_adamw(p.size, _p(p), _p(g), _p(m), _p(v), _p(lr), lr_scale, beta1, beta2, eps, weight_decay, step)


def lr_scale(t: int) -> float:
    return lib().orc_lr_scale(int(t))


def cache_bytes(n: int) -> int:
    return lib().orc_cache_bytes(int(n))
