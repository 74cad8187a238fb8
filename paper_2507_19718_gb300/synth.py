"""Seeded synthetic inputs shaped like the GSCache workloads.

This module only *draws* inputs: Gaussian cache parameters, density volumes,
transfer functions, light set-ups, camera poses and target images.  It holds
none of the method's arithmetic (no projection, compositing, tracking or
optimisation), so both the CUDA path and the CPU oracle may take their inputs
from here.

Every generator is deterministic in its ``seed``.  The shapes and value
distributions follow the paper's setting (Sec. 4.1: 300k-point caches split
into levels of N/2^i, FP32 parameters as in Table 3, volumes mapped through a
predefined 1D transfer function, 1 spp, screen-filling camera paths).  The
paper's six measured volume datasets (Table 1) are not available, so blob and
fBm volumes of the same grid sizes stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20250726

# Packed per-Gaussian record (16 FP32 = 64 B): the paper's 14 attributes
# (Table 3: position 3, rotation 4, colour 3, scale 3, opacity 1) plus two pads
# so that every record is four aligned float4 loads.
SLOT_MEAN = slice(0, 3)
SLOT_OPACITY = 3
SLOT_LOGSCALE = slice(4, 7)
SLOT_QUAT = slice(8, 12)
SLOT_COLOR = slice(12, 15)
PAD_SLOTS = (7, 15)
RECORD_FLOATS = 16


def gaussians(n: int, seed: int, lo: float = 0.0, hi: float = 1.0,
              logscale_mean: float = -3.0, logscale_std: float = 0.5) -> np.ndarray:
    """``n`` anisotropic Gaussians as an (n, 16) float32 packed array.

    means ~ U[lo, hi]^3, log-scales ~ N(-3, 0.5), rotations = normalised
    N(0, 1)^4 quaternions (w, x, y, z), opacity logits ~ N(0, 1), RGB ~ U[0, 1].
    """
    rng = np.random.default_rng(seed)
    p = np.zeros((n, RECORD_FLOATS), np.float64)
    p[:, SLOT_MEAN] = rng.uniform(lo, hi, (n, 3))
    p[:, SLOT_OPACITY] = rng.normal(0.0, 1.0, n)
    p[:, SLOT_LOGSCALE] = rng.normal(logscale_mean, logscale_std, (n, 3))
    q = rng.normal(0.0, 1.0, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    p[:, SLOT_QUAT] = q
    p[:, SLOT_COLOR] = rng.uniform(0.0, 1.0, (n, 3))
    return np.ascontiguousarray(p.astype(np.float32))


def level_sizes(total: int, levels: int) -> list[int]:
    """Split ``total`` Gaussians over ``levels`` cache levels in the paper's
    N/2^i proportions (Sec. 3.2), largest first; the sizes sum to ``total``."""
    w = np.array([0.5 ** i for i in range(levels)])
    raw = total * w / w.sum()
    sizes = np.floor(raw).astype(np.int64)
    rem = total - int(sizes.sum())
    order = np.argsort(-(raw - sizes))
    for i in range(rem):
        sizes[order[i]] += 1
    return [int(s) for s in sizes]


# --------------------------------------------------------------------------
# volumes


def blob_volume(res: int, n_blobs: int, seed: int, peak: float = 20.0,
                sigma_lo: float = 0.05, sigma_hi: float = 0.15) -> np.ndarray:
    """Sum of isotropic Gaussian blobs sampled on a node-centred res^3 grid
    over [0, 1]^3 (voxel i at i / (res - 1)); array layout [z][y][x]."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0.0, 1.0, (n_blobs, 3))
    sig = rng.uniform(sigma_lo, sigma_hi, n_blobs)
    x = np.linspace(0.0, 1.0, res)
    grid = np.zeros((res, res, res), np.float64)
    for (cx, cy, cz), s in zip(centers, sig):
        gx = np.exp(-((x - cx) ** 2) / (2 * s * s))
        gy = np.exp(-((x - cy) ** 2) / (2 * s * s))
        gz = np.exp(-((x - cz) ** 2) / (2 * s * s))
        grid += peak * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return np.ascontiguousarray(grid.astype(np.float32))


def _hash_lattice(ix, iy, iz, seed):
    # 32-bit integer hash of lattice coordinates -> [0, 1)
    h = (ix.astype(np.uint64) * np.uint64(73856093)) ^ (iy.astype(np.uint64) * np.uint64(19349663)) \
        ^ (iz.astype(np.uint64) * np.uint64(83492791)) ^ np.uint64(seed & 0xFFFFFFFF)
    h = h & np.uint64(0xFFFFFFFF)
    h = (h ^ (h >> np.uint64(16))) * np.uint64(0x7FEB352D) & np.uint64(0xFFFFFFFF)
    h = (h ^ (h >> np.uint64(15))) * np.uint64(0x846CA68B) & np.uint64(0xFFFFFFFF)
    h = h ^ (h >> np.uint64(16))
    return (h & np.uint64(0xFFFFFF)).astype(np.float64) / float(1 << 24)


def _value_noise(res: int, freq: float, seed: int) -> np.ndarray:
    """Value noise: hashed lattice values at integer points of x * freq,
    smoothstep-interpolated along each axis (separably, axis by axis)."""
    x = np.linspace(0.0, 1.0, res) * freq
    i0 = np.floor(x).astype(np.int64)
    f = x - i0
    f = f * f * (3 - 2 * f)
    n = int(i0.max()) + 2
    lat = np.arange(n)
    L = _hash_lattice(lat[None, None, :], lat[None, :, None], lat[:, None, None], seed)  # [z][y][x]
    L = L[:, :, i0] * (1 - f)[None, None, :] + L[:, :, i0 + 1] * f[None, None, :]
    L = L[:, i0, :] * (1 - f)[None, :, None] + L[:, i0 + 1, :] * f[None, :, None]
    L = L[i0, :, :] * (1 - f)[:, None, None] + L[i0 + 1, :, :] * f[:, None, None]
    return L


def fbm_volume(res: int, n_blobs: int, seed: int, peak: float = 20.0, octaves: int = 4,
               base_freq: float = 4.0, lacunarity: float = 2.0, gain: float = 0.5,
               amplitude: float = 0.3) -> np.ndarray:
    """Blob volume plus ``octaves`` of hashed value-noise fBm (amplitude
    ``amplitude * peak``), clamped at 0; layout [z][y][x]."""
    grid = blob_volume(res, n_blobs, seed, peak).astype(np.float64)
    noise = np.zeros_like(grid)
    amp, freq = 1.0, base_freq
    for o in range(octaves):
        noise += amp * (2.0 * _value_noise(res, freq, seed * 31 + o) - 1.0)
        amp *= gain
        freq *= lacunarity
    grid += amplitude * peak * noise
    return np.ascontiguousarray(np.maximum(grid, 0.0).astype(np.float32))


def homogeneous_volume(res: int, value: float) -> np.ndarray:
    return np.full((res, res, res), value, np.float32)


def transfer_function(n_points: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Piecewise-linear RGBA transfer function with control points at evenly
    spaced normalised densities; RGBA ~ U[0, 1], opacity forced to 0 at s = 0."""
    rng = np.random.default_rng(seed)
    pos = np.linspace(0.0, 1.0, n_points).astype(np.float32)
    rgba = rng.uniform(0.0, 1.0, (n_points, 4)).astype(np.float32)
    rgba[0, 3] = 0.0
    return pos, np.ascontiguousarray(rgba)


@dataclass
class Scene:
    """Everything the tracer needs besides the camera (plain data)."""
    density: np.ndarray               # [nz][ny][nx] float32
    density_max: float = 20.0         # s = clamp(d / density_max, 0, 1)
    sigma_max: float = 20.0           # sigma_t = sigma_max * A(s)
    albedo: float = 0.8
    tf_pos: np.ndarray = field(default_factory=lambda: np.array([0.0, 1.0], np.float32))
    tf_rgba: np.ndarray = field(default_factory=lambda: np.array([[1, 1, 1, 0], [1, 1, 1, 1]], np.float32))
    light_dir: np.ndarray = field(default_factory=lambda: np.array([0.0, 0.0, 1.0], np.float32))
    light_radiance: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))
    env_radiance: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))
    # spherical area lights outside the box: (centre (3,), radius, radiance (3,))
    spheres: list = field(default_factory=list)


def two_sphere_lights(radiance: float = 40.0, radius: float = 0.15, distance: float = 1.6,
                      elevation_deg: float = 45.0, azimuths_deg=(-60.0, 60.0)):
    """The paper's two-point lighting (Sec. 4.3: two small spherical area
    lights outside the volume), placed at `distance` from the box centre at
    the given azimuths (around z) and elevation; sizes and radiance are not
    given in the paper and are chosen here (irradiance at the centre about
    radiance * pi radius^2 / distance^2 = 1.1 each)."""
    out = []
    el = np.radians(elevation_deg)
    for az in azimuths_deg:
        a = np.radians(az)
        c = 0.5 + distance * np.array([np.cos(el) * np.cos(a), np.cos(el) * np.sin(a), np.sin(el)])
        out.append((c.astype(np.float32), float(radius), np.full(3, radiance, np.float32)))
    return out


def unit(v) -> np.ndarray:
    v = np.asarray(v, np.float64)
    return (v / np.linalg.norm(v)).astype(np.float32)


def scene_tiny(seed: int = BASE_SEED) -> Scene:
    """64^3 grid of 8 blobs, 4-point TF, directional light along (1,1,1) with
    radiance 3, no environment, albedo 0.8."""
    pos, rgba = transfer_function(4, seed + 1)
    return Scene(density=blob_volume(64, 8, seed), tf_pos=pos, tf_rgba=rgba,
                 light_dir=unit([1, 1, 1]), light_radiance=np.full(3, 3.0, np.float32),
                 env_radiance=np.zeros(3, np.float32))


def scene_frame(res: int = 256, seed: int = BASE_SEED + 1) -> Scene:
    """res^3 grid of 64 blobs + 4-octave fBm, 8-point TF, directional light
    (radiance 3) plus constant environment 0.3."""
    pos, rgba = transfer_function(8, seed + 1)
    return Scene(density=fbm_volume(res, 64, seed), tf_pos=pos, tf_rgba=rgba,
                 light_dir=unit([1, 1, 1]), light_radiance=np.full(3, 3.0, np.float32),
                 env_radiance=np.full(3, 0.3, np.float32))


# --------------------------------------------------------------------------
# cameras


@dataclass
class Camera:
    """Pinhole camera.  ``R`` rows are the camera's right, down and forward
    axes in world space (world -> camera rotation); x_cam = R x_world + t."""
    R: np.ndarray      # (3, 3) float32
    t: np.ndarray      # (3,) float32
    pos: np.ndarray    # (3,) float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def packed(self) -> np.ndarray:
        """R[9], t[3], pos[3], fx, fy, cx, cy as 19 float32."""
        return np.concatenate([self.R.reshape(-1), self.t, self.pos,
                               np.array([self.fx, self.fy, self.cx, self.cy], np.float32)]).astype(np.float32)


def look_at(pos, target, up, width: int, height: int, fov_y_deg: float = 45.0) -> Camera:
    pos = np.asarray(pos, np.float64)
    f = np.asarray(target, np.float64) - pos
    f /= np.linalg.norm(f)
    right = np.cross(f, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f])
    t = -R @ pos
    fy = height / (2.0 * math.tan(math.radians(fov_y_deg) / 2.0))
    return Camera(R=R.astype(np.float32), t=t.astype(np.float32), pos=pos.astype(np.float32),
                  fx=float(np.float32(fy)), fy=float(np.float32(fy)),
                  cx=float(width) / 2.0, cy=float(height) / 2.0, width=width, height=height)


def orbit_camera(width: int, height: int, angle_deg: float, radius: float = 2.2,
                 elevation_deg: float = 15.0, fov_y_deg: float = 45.0,
                 center=(0.5, 0.5, 0.5)) -> Camera:
    """Camera on a z-up orbit around ``center`` looking at it."""
    a, e = math.radians(angle_deg), math.radians(elevation_deg)
    c = np.asarray(center, np.float64)
    pos = c + radius * np.array([math.cos(a) * math.cos(e), math.sin(a) * math.cos(e), math.sin(e)])
    return look_at(pos, c, (0.0, 0.0, 1.0), width, height, fov_y_deg)


def axis_camera(width: int, height: int, z: float = -1.0, f: float | None = None,
                fov_y_deg: float = 45.0) -> Camera:
    """Camera at (0.5, 0.5, z) looking along +z with identity rotation
    (camera axes = world axes); used by closed-form checks."""
    fy = height / (2.0 * math.tan(math.radians(fov_y_deg) / 2.0)) if f is None else f
    pos = np.array([0.5, 0.5, z], np.float64)
    R = np.eye(3)
    return Camera(R=R.astype(np.float32), t=(-pos).astype(np.float32), pos=pos.astype(np.float32),
                  fx=float(fy), fy=float(fy), cx=width / 2.0, cy=height / 2.0, width=width, height=height)


# --------------------------------------------------------------------------
# targets and noise


def uniform_image(c: int, h: int, w: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.0, 1.0, (c, h, w)).astype(np.float32)


def smooth_noisy_image(c: int, h: int, w: int, seed: int, noise_std: float = 0.05) -> np.ndarray:
    """A smooth seeded colour field plus N(0, noise_std^2) noise per element."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    out = np.empty((c, h, w), np.float64)
    for ch in range(c):
        kx, ky, ph = rng.uniform(0.5, 3.0), rng.uniform(0.5, 3.0), rng.uniform(0, 2 * math.pi)
        out[ch] = 0.5 + 0.4 * np.sin(2 * math.pi * (kx * xx / w + ky * yy / h) + ph)
    out += rng.normal(0.0, noise_std, out.shape)
    return out.astype(np.float32)
