"""Pins of the oracle volume path tracer (Sec. 3.1 Eq. 1, Sec. 3.2, Sec. 3.3,
Sec. 3.5).

Closed forms: sigma_t of a linear density ramp through a piecewise-linear TF;
Beer-Lambert exp(-sigma l) for the escape probability in a homogeneous
medium; the single-scattering value of a homogeneous slab lit by a
directional light.  Invariants: the white furnace (albedo 1, environment
only, unbounded bounces => every pixel's expectation is L_env); delta and
ratio tracking agree with exp(-integral sigma) by quadrature; the target
buffers and the primary-escape term sum to the image; Algorithm 1 with
C -> infinity is the identity.  Algorithm 1's termination into the cache:
closed forms at C -> 0+, after one roulette survival (the escape probability
of a dense half-space), and without roulette from Tr = 0.9 up.
"""
import math

import numpy as np
import pytest

from paper_2507_19718_gb300 import synth


def _homog_scene(sigma, rgb=(1.0, 1.0, 1.0), albedo=0.8, light=(0, 0, 0), ldir=(1, 0, 0), env=(0, 0, 0)):
    rgba = np.array([[*rgb, 0.0], [*rgb, 1.0]], np.float32)
    return synth.Scene(density=synth.homogeneous_volume(8, 20.0), density_max=20.0, sigma_max=sigma,
                       albedo=albedo, tf_pos=np.array([0.0, 1.0], np.float32), tf_rgba=rgba,
                       light_dir=synth.unit(ldir), light_radiance=np.array(light, np.float32),
                       env_radiance=np.array(env, np.float32))


def _far_cam(n=4, dist=100.0, f=40000.0):
    """Nearly orthographic camera looking along +z at the box centre."""
    cam = synth.axis_camera(n, n, z=-dist)
    cam.fx = cam.fy = f
    return cam


def _ratio_check(values, expected, k=4.5):
    r = np.asarray(values).ravel() / np.asarray(expected).ravel()
    se = r.std(ddof=1) / math.sqrt(r.size)
    assert abs(r.mean() - 1.0) <= k * se + 1e-3, (r.mean(), se)


def test_sigma_t_of_linear_ramp(orc):
    """Trilinear interpolation reproduces a linear density exactly; the TF maps
    it piecewise linearly."""
    n = 17
    x = np.linspace(0, 1, n)
    grid = np.broadcast_to(20.0 * x[None, None, :], (n, n, n)).astype(np.float32).copy()
    tf_pos = np.array([0.0, 0.5, 1.0], np.float32)
    tf_rgba = np.array([[1, 1, 1, 0.0], [1, 1, 1, 1.0], [1, 1, 1, 0.2]], np.float32)
    sc = synth.Scene(density=grid, density_max=20.0, sigma_max=7.0, tf_pos=tf_pos, tf_rgba=tf_rgba)
    pts = np.random.default_rng(0).uniform(0, 1, (500, 3))
    got = orc.sigma_t(sc, pts)
    s = pts[:, 0]
    A = np.where(s < 0.5, s / 0.5, 1.0 + (s - 0.5) / 0.5 * (0.2 - 1.0))
    np.testing.assert_allclose(got, 7.0 * A, rtol=2e-6, atol=2e-6)


@pytest.mark.parametrize("precision", [64, 32])
def test_beer_lambert(orc, precision):
    sigma = 2.0
    sc = _homog_scene(sigma, albedo=0.0, env=(1.0, 1.0, 1.0))
    cam = _far_cam()
    _, img = orc.trace(sc, cam, spp=2048, max_bounces=1, levels=1, seed=7, precision=precision)
    # chord through the unit box along the (almost exactly +z) pixel rays
    expected = math.exp(-sigma * 1.0)
    p = img[0].mean()
    se = math.sqrt(expected * (1 - expected) / (16 * 2048))
    assert abs(p - expected) < 4.5 * se, (p, expected, se)
    np.testing.assert_array_equal(img[0], img[1])


def test_single_scatter_directional_light(orc):
    """B = 1, homogeneous sigma, albedo rgb a, directional light along +x:
    E[pixel] = (1 - e^{-sigma l}) a L_d / (4 pi) e^{-sigma (1 - x)}."""
    sigma, Ld = 1.5, 3.0
    rgb = (1.0, 0.5, 0.25)
    sc = _homog_scene(sigma, rgb=rgb, albedo=0.8, light=(Ld, Ld, Ld), ldir=(1, 0, 0))
    cam = _far_cam()
    _, img = orc.trace(sc, cam, spp=4096, max_bounces=1, levels=1, seed=9)
    ii = np.arange(4) + 0.5
    x = 0.5 + (ii - cam.cx) / cam.fx * 100.0
    base = (1 - math.exp(-sigma)) * Ld / (4 * math.pi) * np.exp(-sigma * (1 - x))
    for ch, c in enumerate(rgb):
        exp_img = np.broadcast_to(0.8 * c * base[None, :], (4, 4))
        _ratio_check(img[ch], exp_img)


def test_white_furnace(orc):
    """Albedo 1, a constant environment as the only light and no bounce limit:
    every pixel's expectation is L_env (the NEE terms telescope)."""
    sc = _homog_scene(3.0, rgb=(1, 1, 1), albedo=1.0, env=(1.0, 1.0, 1.0))
    cam = synth.orbit_camera(12, 12, 20.0)
    _, img, lens = orc.trace(sc, cam, spp=256, max_bounces=100000, levels=1, seed=3, lengths=True)
    assert lens.max() > 5  # paths really scatter many times
    inside = (lens > 0).mean(axis=2) > 0.5
    assert inside.sum() > 20
    _ratio_check(img[0][inside], np.ones(inside.sum()))
    np.testing.assert_allclose(img[0][~inside].mean(), 1.0, atol=0.05)


def test_delta_and_ratio_tracking_agree_with_quadrature(orc):
    sc = synth.scene_tiny()
    sc.sigma_max = 4.0
    o = np.array([-0.2, 0.31, 0.42])
    d = np.array([1.0, 0.21, 0.13])
    d /= np.linalg.norm(d)
    # chord through the unit box, then exp(-int sigma) by the trapezoid rule
    t0 = max(np.max(np.minimum((0 - o) / d, (1 - o) / d)), 0.0)
    t1 = np.min(np.maximum((0 - o) / d, (1 - o) / d))
    ts = np.linspace(t0, t1, 20001)
    sig = orc.sigma_t(sc, o[None, :] + ts[:, None] * d[None, :])
    tau = np.trapezoid(sig, ts)
    T = math.exp(-tau)
    assert 0.05 < T < 0.95
    n = 200000
    dt = orc.transmittance("delta", sc, o, d, n, seed=1)
    rt = orc.transmittance("ratio", sc, o, d, n, seed=2)
    assert abs(dt.mean() - T) < 4.5 * dt.std() / math.sqrt(n)
    assert abs(rt.mean() - T) < 4.5 * rt.std() / math.sqrt(n)
    assert rt.std() < dt.std()  # ratio tracking is the lower-variance estimator


def test_buffers_and_escapes_sum_to_image(orc):
    """Each sample writes its NEE radiance to the buffer of its length, so with
    K >= B the buffers plus L_env times the primary-escape fraction equal the
    image (Sec. 3.5: at most one buffer entry per sample)."""
    sc = synth.scene_tiny()
    sc.env_radiance = np.array([0.2, 0.3, 0.4], np.float32)
    cam = synth.orbit_camera(24, 20, 35.0)
    tg, img, lens = orc.trace(sc, cam, spp=3, max_bounces=3, levels=3, seed=5, lengths=True)
    esc = (lens == 0).mean(axis=2)
    recon = tg.sum(0) + sc.env_radiance[:, None, None].astype(np.float64) * esc[None]
    np.testing.assert_allclose(recon, img, rtol=1e-12, atol=1e-15)
    assert tg[0].max() > 0 and tg[1].max() > 0
    # K < B: long paths write nothing
    tg2, _ = orc.trace(sc, cam, spp=3, max_bounces=3, levels=1, seed=5)
    np.testing.assert_array_equal(tg2[0], tg[0])


def test_algorithm1_with_infinite_C_is_identity(orc):
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(20, 16, 60.0)
    cache = synth.uniform_image(4 * 3, 16, 20, 77).reshape(4, 3, 16, 20)
    a = orc.trace(sc, cam, spp=2, max_bounces=4, levels=4, seed=11, C=0.0, cache=cache, precision=32)
    b = orc.trace(sc, cam, spp=2, max_bounces=4, levels=4, seed=11, C=1e30, cache=cache, precision=32)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    c = orc.trace(sc, cam, spp=2, max_bounces=4, levels=4, seed=11, C=0.5, cache=cache, precision=32)
    assert not np.array_equal(a[1], c[1])
    assert np.all(np.isfinite(c[0])) and np.all(np.isfinite(c[1]))


def _const_cache(levels, h, w, per_level):
    """Cache images: level k holds the constant colour per_level[k]."""
    c = np.zeros((levels, 3, h, w), np.float32)
    for k, rgb in enumerate(per_level):
        c[k] = np.asarray(rgb, np.float32)[:, None, None]
    return c


# escape probability of a path scattered isotropically at the exponentially
# distributed depth of a beam entering a half-space at normal incidence:
# 1/2 int_0^1 mu / (1 + mu) dmu
P_ESC_HALF_SPACE = 0.5 * (1.0 - math.log(2.0))


@pytest.mark.parametrize("precision", [64, 32])
def test_algorithm1_with_vanishing_C_terminates_at_the_first_vertex(orc, precision):
    """C -> 0+: Tr = 0 at the first vertex, so every path that collides ends
    there in the cache's level 1 (index 0, not divided: no earlier survival)
    and every primary escape shows the environment:
    E[pixel] = e^{-sigma} L_env + (1 - e^{-sigma}) cache_1."""
    sigma, env = 1.0, 0.7
    sc = _homog_scene(sigma, albedo=0.8, env=(env, env, env))
    cam = _far_cam()
    c1, c2 = (0.3, 0.5, 0.9), (5.0, 6.0, 7.0)
    cache = _const_cache(2, 4, 4, [c1, c2])
    _, img = orc.trace(sc, cam, spp=4096, max_bounces=4, levels=2, seed=21, C=1e-30, cache=cache,
                       precision=precision)
    pe = math.exp(-sigma)
    for ch in range(3):
        _ratio_check(img[ch], np.full((4, 4), pe * env + (1 - pe) * c1[ch]))


@pytest.mark.parametrize("precision", [64, 32])
def test_algorithm1_survival_weight_and_escape_into_the_cache(orc, precision):
    """A dense half-space (sigma = 200 in the unit box), no lights, B = 2, and
    Tr = C lum(albedo) = 0.3 at the first vertex: a path ends there in the
    cache with probability 1 - Tr (value cache_1); it survives with
    probability Tr, beta = Tr, and then either escapes with no radiance
    (value cache_1 / beta) or collides at the bounce limit (value 0):
    E[pixel] = cache_1 (1 - Tr + P_esc), P_esc = (1 - ln 2) / 2.  The TF colour
    is not grey, so Tr also pins the Rec. 709 luminance of the throughput."""
    rgb = (1.0, 0.5, 0.25)
    sc = _homog_scene(200.0, rgb=rgb, albedo=0.8)
    cam = _far_cam()
    c1, c2 = (0.3, 0.5, 0.9), (5.0, 6.0, 7.0)
    cache = _const_cache(2, 4, 4, [c1, c2])
    Tr = 0.3
    lum = 0.8 * (0.2126 * rgb[0] + 0.7152 * rgb[1] + 0.0722 * rgb[2])
    _, img = orc.trace(sc, cam, spp=4096, max_bounces=2, levels=2, seed=22, C=Tr / lum, cache=cache,
                       precision=precision)
    for ch in range(3):
        _ratio_check(img[ch], np.full((4, 4), c1[ch] * (1 - Tr + P_ESC_HALF_SPACE)))


@pytest.mark.parametrize("precision", [64, 32])
def test_algorithm1_no_roulette_from_tr_09(orc, precision):
    """As above with Tr = 0.95 >= 0.9: no roulette at the first vertex, so
    only the escaped paths end in the cache, undivided:
    E[pixel] = cache_1 P_esc."""
    sc = _homog_scene(200.0, albedo=0.8)
    cam = _far_cam()
    c1, c2 = (0.3, 0.5, 0.9), (5.0, 6.0, 7.0)
    cache = _const_cache(2, 4, 4, [c1, c2])
    _, img = orc.trace(sc, cam, spp=4096, max_bounces=2, levels=2, seed=23, C=0.95 / 0.8, cache=cache,
                       precision=precision)
    for ch in range(3):
        _ratio_check(img[ch], np.full((4, 4), c1[ch] * P_ESC_HALF_SPACE))


def test_fp32_mirror_tracks_fp64(orc):
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(32, 32, 15.0)
    t64, i64 = orc.trace(sc, cam, spp=4, max_bounces=4, levels=4, seed=20250726, precision=64)
    t32, i32 = orc.trace(sc, cam, spp=4, max_bounces=4, levels=4, seed=20250726, precision=32)
    diff = np.abs(i64 - i32)
    # same Philox streams: almost every pixel follows the same paths
    assert np.median(diff) < 1e-5
    assert abs(i64.mean() - i32.mean()) < 0.02 * i64.mean()
    assert i64.max() > 0


def test_seed_and_frame_select_streams(orc):
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(12, 10, 5.0)
    a = orc.trace(sc, cam, spp=1, max_bounces=4, levels=2, seed=1, frame=0, precision=32)[1]
    b = orc.trace(sc, cam, spp=1, max_bounces=4, levels=2, seed=1, frame=0, precision=32)[1]
    c = orc.trace(sc, cam, spp=1, max_bounces=4, levels=2, seed=1, frame=1, precision=32)[1]
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)


def test_single_scatter_small_far_sphere_light(orc):
    """The same slab lit by a small spherical area light far along +x
    (Sec. 4.3's light type): the cone estimate's expectation is L_e T
    (1 - cos theta_max) / 2 per vertex, i.e. the directional closed form with
    L_d = 2 pi (1 - cos theta_max) L_e (to the 1e-3 variation of theta_max
    over the box at distance 1000)."""
    sigma, Ld = 1.5, 3.0
    rgb = (1.0, 0.5, 0.25)
    D, rad = 1000.0, 20.0
    one_minus_cos = 1.0 - math.sqrt(1.0 - (rad / D) ** 2)
    Le = Ld / (2 * math.pi * one_minus_cos)
    sc = _homog_scene(sigma, rgb=rgb, albedo=0.8)
    sc.spheres = [(np.array([0.5 + D, 0.5, 0.5], np.float32), rad, np.full(3, Le, np.float32))]
    cam = _far_cam()
    _, img = orc.trace(sc, cam, spp=4096, max_bounces=1, levels=1, seed=19)
    ii = np.arange(4) + 0.5
    x = 0.5 + (ii - cam.cx) / cam.fx * 100.0
    base = (1 - math.exp(-sigma)) * Ld / (4 * math.pi) * np.exp(-sigma * (1 - x))
    for ch, c in enumerate(rgb):
        r = img[ch].ravel() / np.broadcast_to(0.8 * c * base[None, :], (4, 4)).ravel()
        se = r.std(ddof=1) / math.sqrt(r.size)
        assert abs(r.mean() - 1.0) <= 4.5 * se + 2e-3, (r.mean(), se)


def test_sphere_lights_add_linearly(orc):
    """Two sphere lights together equal the sum of each alone (same streams
    are not shared, so in expectation): NEE terms are additive."""
    sc = synth.scene_tiny()
    sc.light_radiance = np.zeros(3, np.float32)
    lights = synth.two_sphere_lights()
    cam = synth.orbit_camera(24, 24, 10.0)
    imgs = []
    for sph in ([lights[0]], [lights[1]], lights):
        sc.spheres = sph
        _, img = orc.trace(sc, cam, spp=512, max_bounces=2, levels=2, seed=23)
        imgs.append(img)
    both, a, b = imgs[2], imgs[0], imgs[1]
    assert a.mean() > 0 and b.mean() > 0
    assert abs(both.mean() - (a.mean() + b.mean())) < 0.03 * both.mean()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("rgb,albedo,tr1", [((1.0, 1.0, 1.0), 0.8, 0.5), ((1.2, 1.2, 1.2), 1.0, 0.85)])
def test_algorithm1_per_call_reading_keeps_only_its_own_division(orc, precision, rgb, albedo, tr1):
    """The per-call reading of Algorithm 1 (every call starts from the
    product of the albedos and divides by its own Tr + eps only) against the
    cumulative one, in a grey homogeneous medium, where Tr_n = C a^n is the
    same at every path's n-th vertex.  Both readings draw the same numbers, so
    every sample takes the same path; with B = 3 they differ only in the
    next-event weight of the third vertex: cumulative a^3 / ((Tr_1 + eps)
    (Tr_2 + eps)), per call a^3 / (Tr_2 + eps) when the second call divides
    (first case, Tr_2 = 0.4), a^3 when it does not (second case, a = 1.2:
    Tr_2 = 1 >= 0.9, so the second call returns the undivided product).
    Either way the per-call weight is the cumulative one times Tr_1 + eps, so
    the summed target buffers satisfy, per pixel,
    T_call(B=3) = T(B=2) + (Tr_1 + eps) (T_cum(B=3) - T(B=2)),
    where B = 2 keeps the first two vertices, the same in both readings."""
    sc = _homog_scene(3.0, rgb=rgb, albedo=albedo, light=(2.0, 2.0, 2.0), ldir=(0.3, 0.4, -0.866),
                      env=(0.4, 0.4, 0.4))
    cam = _far_cam()
    cache = _const_cache(3, 4, 4, [(0.3, 0.5, 0.9)] * 3)
    a = albedo * rgb[0]
    C = tr1 / a
    eps = 1e-6

    def summed(B, mode):
        t, _ = orc.trace(sc, cam, spp=64, max_bounces=B, levels=3, seed=31, C=C, eps=eps, cache=cache,
                         precision=precision, tr_out=mode)
        return t.sum(0)
    b2 = summed(2, 0)
    np.testing.assert_array_equal(summed(2, 1), b2)
    cum3, call3 = summed(3, 0), summed(3, 1)
    assert np.all(cum3 >= b2 * (1 - 1e-6)) and (cum3 - b2).sum() > 0.1 * b2.sum()  # the third vertex contributes
    # Tr_1 as the tracer forms it from its FP32 inputs (albedo, TF colour, C)
    a1 = float(np.float32(albedo)) * float(np.float32(rgb[0]))
    tr1_exact = float(np.float32(C)) * ((0.2126 * a1 + 0.7152 * a1) + 0.0722 * a1)
    rtol = 1e-12 if precision == 64 else 2e-6
    np.testing.assert_allclose(call3, b2 + (tr1_exact + eps) * (cum3 - b2), rtol=rtol)
