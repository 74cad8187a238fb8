"""Pins of the oracle rasterizer (Gaussian splatting of one cache level,
Sec. 3.1) and of its analytic backward (the inverse splatting step, Sec. 3.5).

The forward is pinned by closed forms of special cases (an isotropic Gaussian
on the optical axis, a rotated anisotropic one, opaque fronts, the near
plane), by compositing invariants (associativity of front and back groups,
invariance to input order) and by Table 3's byte counts; the backward by
central finite differences of the FP64 forward for every parameter kind.
"""
import math
import os

import numpy as np
import pytest

from paper_2507_19718_gb300 import synth

CFG = dict(alpha_max=0.99, alpha_min=1 / 255, T_min=1e-4, near=0.2, dilation=0.3)


def _one(mean, logscale, quat, logit, rgb):
    p = np.zeros((1, 16), np.float32)
    p[0, 0:3] = mean
    p[0, 3] = logit
    p[0, 4:7] = logscale
    p[0, 8:12] = quat
    p[0, 12:15] = rgb
    return p


def _axis_cam(W=65, H=65, fx=80.0, fy=60.0):
    cam = synth.axis_camera(W, H, z=-1.0)
    cam.fx, cam.fy = fx, fy
    cam.cx, cam.cy = W / 2.0, H / 2.0
    return cam


def test_isotropic_gaussian_on_axis_closed_form(orc):
    """A sphere-shaped Gaussian of std s at depth z on the optical axis images
    to a 2D Gaussian with std (f s / z) per axis, widened by the 0.3 px^2
    dilation; its peak alpha is its opacity sigmoid(o)."""
    cam = _axis_cam()
    s, zc, logit = 0.05, 1.5, 0.4
    tz = zc + 1.0
    p = _one([0.5, 0.5, zc], [math.log(s)] * 3, [1, 0, 0, 0], logit, [1.0, 0.5, 0.25])
    img, marg, ncon, _ = orc.render(p, cam, CFG)
    logit, s, tz = float(p[0, 3]), math.exp(float(p[0, 4])), float(p[0, 2]) + 1.0
    op = 1 / (1 + math.exp(-logit))
    vx = (cam.fx * s / tz) ** 2 + 0.3
    vy = (cam.fy * s / tz) ** 2 + 0.3
    jj, ii = np.mgrid[0:65, 0:65]
    dx, dy = ii + 0.5 - 32.5, jj + 0.5 - 32.5
    alpha = op * np.exp(-0.5 * (dx * dx / vx + dy * dy / vy))
    alpha = np.where(alpha >= 1 / 255, np.minimum(alpha, 0.99), 0.0)
    assert img[0, 32, 32] == pytest.approx(op, rel=1e-12)
    for ch, c in enumerate([1.0, 0.5, 0.25]):
        np.testing.assert_allclose(img[ch], c * alpha, rtol=1e-10, atol=1e-14)
    assert ncon.max() == 1


def test_off_axis_isotropic_gaussian_closed_form(orc):
    """Off the axis, an isotropic 3D Gaussian images with covariance
    s^2 J J^T + 0.3 I, J the pinhole Jacobian at its camera-space mean, and is
    centred at the perspective projection of its mean."""
    cam = _axis_cam(W=96, H=80, fx=70.0, fy=90.0)
    mean = np.array([0.8, 0.35, 1.2])
    s = 0.06
    p = _one(mean, [math.log(s)] * 3, [0.3, 0, 0, 0], 1.0, [1, 1, 1])
    t = p[0, 0:3].astype(np.float64) + cam.t.astype(np.float64)
    s = math.exp(float(p[0, 4]))
    img, _, _, _ = orc.render(p, cam, CFG)
    J = np.array([[cam.fx / t[2], 0, -cam.fx * t[0] / t[2] ** 2], [0, cam.fy / t[2], -cam.fy * t[1] / t[2] ** 2]])
    cov = s * s * J @ J.T + 0.3 * np.eye(2)
    mu = np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])
    jj, ii = np.mgrid[0:80, 0:96]
    d = np.stack([ii + 0.5 - mu[0], jj + 0.5 - mu[1]], -1)
    q = np.einsum("...i,ij,...j->...", d, np.linalg.inv(cov), d)
    alpha = (1 / (1 + math.exp(-1.0))) * np.exp(-0.5 * q)
    alpha = np.where(alpha >= 1 / 255, np.minimum(alpha, 0.99), 0.0)
    np.testing.assert_allclose(img[1], alpha, rtol=1e-9, atol=1e-13)


def test_rotated_anisotropic_gaussian_axes(orc):
    """q = (cos th/2, 0, 0, sin th/2) turns the Gaussian's x axis to
    (cos th, sin th) in the image (x right, y down): along it the std is
    f s1 / z, across it f s2 / z (plus dilation)."""
    cam = _axis_cam(W=65, H=65, fx=90.0, fy=90.0)
    th = math.atan2(3.0, 4.0)
    s1, s2, zc = 0.09, 0.03, 1.0
    tz = zc + 1.0
    p = _one([0.5, 0.5, zc], [math.log(s1), math.log(s2), math.log(0.05)],
             [math.cos(th / 2), 0, 0, math.sin(th / 2)], 3.0, [1, 1, 1])
    img, _, _, _ = orc.render(p, cam, CFG)
    op = min(0.99, 1 / (1 + math.exp(-3.0)))
    s1, s2 = math.exp(float(p[0, 4])), math.exp(float(p[0, 5]))
    v1 = (90.0 * s1 / tz) ** 2 + 0.3
    v2 = (90.0 * s2 / tz) ** 2 + 0.3
    for k in range(1, 4):
        # along (0.8, 0.6): pixel offset (4k, 3k), distance 5k
        a_along = op * math.exp(-0.5 * (5 * k) ** 2 / v1)
        a_across = op * math.exp(-0.5 * (5 * k) ** 2 / v2)
        got_along = img[0, 32 + 3 * k, 32 + 4 * k]
        got_across = img[0, 32 + 4 * k, 32 - 3 * k]
        assert got_along == pytest.approx(a_along if a_along >= 1 / 255 else 0.0, rel=1e-9, abs=1e-14)
        assert got_across == pytest.approx(a_across if a_across >= 1 / 255 else 0.0, rel=1e-9, abs=1e-14)


def test_opaque_fronts_occlude(orc):
    """Front-to-back compositing with alpha clamped to alpha_max: the second
    layer is weighted by (1 - alpha_max); a third layer would drive T below
    T_min, so the walk stops and nothing behind contributes."""
    cam = _axis_cam(W=33, H=33, fx=40.0, fy=40.0)
    cfg = dict(CFG, alpha_max=0.98)
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]]
    p = np.concatenate([_one([0.5, 0.5, z], [math.log(0.3)] * 3, [1, 0, 0, 0], 12.0, c)
                        for z, c in zip([0.2, 0.4, 0.6, 0.8], cols)])
    img, _, ncon, tfin = orc.render(p, cam, cfg)
    np.testing.assert_allclose(img[:, 16, 16], [0.98, 0.98 * 0.02, 0.0], rtol=1e-12)
    assert ncon[16, 16] == 2
    assert tfin[16, 16] == pytest.approx(0.02 * 0.02, rel=1e-12)
    # the order of the inputs does not matter, only their depth
    img2, _, _, _ = orc.render(p[::-1].copy(), cam, cfg)
    np.testing.assert_array_equal(img, img2)


def test_near_plane_culls(orc):
    cam = _axis_cam(W=33, H=33, fx=40.0, fy=40.0)
    # camera at z = -1: depth 0.1 is in front of the camera but before near = 0.2
    p = _one([0.5, 0.5, -0.9], [math.log(0.2)] * 3, [1, 0, 0, 0], 2.0, [1, 1, 1])
    img, _, _, _ = orc.render(p, cam, CFG)
    assert np.all(img == 0)
    p[0, 2] = -0.7  # depth 0.3
    img, _, _, _ = orc.render(p, cam, CFG)
    assert img.max() > 0.5


def test_front_back_groups_compose(orc):
    """C(A u B) = C(A) + T(A) C(B) when every Gaussian of A lies in front of
    every Gaussian of B (and T stays above T_min); T(A u B) = T(A) T(B)."""
    cam = synth.orbit_camera(48, 40, 30.0)
    rng = np.random.default_rng(11)
    A = synth.gaussians(40, 1, lo=0.35, hi=0.65, logscale_mean=-2.6)
    B = synth.gaussians(40, 2, lo=0.35, hi=0.65, logscale_mean=-2.6)
    # push B far behind A along the view direction
    fwd = cam.R[2].astype(np.float64)
    B[:, 0:3] = (B[:, 0:3] + 1.5 * fwd).astype(np.float32)
    A[:, 3] = rng.normal(-2.5, 0.3, 40)
    B[:, 3] = rng.normal(-2.5, 0.3, 40)
    ia, ma, _, ta = orc.render(A, cam, CFG)
    ib, mb, _, tb = orc.render(B, cam, CFG)
    iab, mab, _, tab = orc.render(np.concatenate([A, B]), cam, CFG)
    assert tab.min() > 1e-3
    np.testing.assert_allclose(iab, ia + ta[None] * ib, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(tab, ta * tb, rtol=1e-12)
    assert ia.max() > 0.02 and ib.max() > 0.01


def test_input_order_invariance(orc):
    cam = synth.orbit_camera(40, 32, 75.0)
    p = synth.gaussians(200, 5, lo=0.2, hi=0.8, logscale_mean=-2.8)
    perm = np.random.default_rng(0).permutation(200)
    i1, _, _, _ = orc.render(p, cam, CFG)
    i2, _, _, _ = orc.render(p[perm], cam, CFG)
    np.testing.assert_array_equal(i1, i2)
    assert i1.max() > 0.1


def test_window_matches_full_frame(orc):
    cam = synth.orbit_camera(40, 32, 10.0)
    p = synth.gaussians(150, 6, lo=0.2, hi=0.8, logscale_mean=-2.8)
    full, _, _, _ = orc.render(p, cam, CFG)
    win, _, _, _ = orc.render(p, cam, CFG, window=(7, 5, 20, 13))
    np.testing.assert_array_equal(win, full[:, 5:18, 7:27])


def test_table3_memory(orc):
    path = os.path.join(os.path.dirname(__file__), "golden", "table3_memory.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            n, b = map(int, line.split())
            assert orc.cache_bytes(n) == b
    assert sum(synth.level_sizes(525000, 3)) == 525000
    assert synth.level_sizes(525000, 3) == [300000, 150000, 75000]


# ----------------------------------------------------------------- backward

def _fd_scene():
    cam = synth.orbit_camera(36, 30, 40.0, radius=2.0)
    p = synth.gaussians(18, 21, lo=0.3, hi=0.7, logscale_mean=-2.4, logscale_std=0.3)
    p[:, 3] = np.random.default_rng(22).normal(-0.5, 0.8, len(p))
    p[3, 12] = -0.2  # one clamped colour channel: its gradient must be 0
    return cam, p


@pytest.mark.parametrize("slot", [0, 1, 2, 3, 4, 5, 6, 8, 9, 10, 11, 12, 13, 14])
def test_backward_matches_finite_differences(orc, slot):
    cam, p = _fd_scene()
    rng = np.random.default_rng(100 + slot)
    W = rng.uniform(-1, 1, (3, cam.height, cam.width))
    grads, _ = orc.render_backward(p, cam, W, CFG)
    _, _, ncon0, _ = orc.render(p, cam, CFG)
    h = 1e-4
    checked = 0
    gmax = np.abs(grads[:, slot]).max()
    for g in range(len(p)):
        pp, pm = p.copy(), p.copy()
        pp[g, slot] = np.float32(p[g, slot] + h)
        pm[g, slot] = np.float32(p[g, slot] - h)
        heff = (np.float64(pp[g, slot]) - np.float64(pm[g, slot])) / 2
        ip, _, ncp, _ = orc.render(pp, cam, CFG)
        im, _, ncm, _ = orc.render(pm, cam, CFG)
        if not (np.array_equal(ncp, ncon0) and np.array_equal(ncm, ncon0)):
            continue  # the perturbation crossed a threshold: not differentiable here
        fd = (np.sum(W * ip) - np.sum(W * im)) / (2 * heff)
        an = grads[g, slot]
        assert abs(fd - an) <= 2e-4 * max(abs(an), 1e-3 * gmax) + 1e-10, (g, slot, fd, an)
        checked += 1
    assert checked >= len(p) // 2
    if slot == 12:
        assert grads[3, 12] == 0.0
    assert gmax > 0


# ----------------------------------------------------------------- frozen decisions

FD_SLOTS = [0, 1, 2, 3, 4, 5, 6, 8, 9, 10, 11, 12, 13, 14]


def _dense_scene():
    """Opaque, overlapping Gaussians: pixels stop at T_min and some alphas sit
    at the alpha_max clamp, so plain differences cross decisions."""
    cam = synth.orbit_camera(40, 32, 25.0, radius=2.0)
    p = synth.gaussians(60, 31, lo=0.35, hi=0.65, logscale_mean=-2.2, logscale_std=0.3)
    p[:, 3] = np.random.default_rng(32).normal(2.5, 1.0, len(p))
    p[::7, 3] = 6.0  # alpha = 0.9975 G: clamped near these means
    p[::7, 4:7] += 1.0
    toward = np.asarray(cam.pos, np.float64) - 0.5
    toward /= np.linalg.norm(toward)
    p[:14:7, 0:3] += (0.3 * toward).astype(np.float32)  # two of them in front of the rest
    return cam, p


def test_frozen_lists_reproduce_the_render(orc):
    cam, p = _dense_scene()
    img, _, ncon, T = orc.render(p, cam, CFG)
    fl = orc.FrozenLists(p, cam, CFG)
    assert np.array_equal(fl.render(p), img)
    assert fl.clamped.any()                         # clamped alphas are frozen too
    assert (T < 1e-3).any()                         # some pixels ran into T_min
    assert int(fl.offsets[-1]) == int(ncon.sum())


def test_frozen_differences_equal_the_backward_for_every_parameter(orc):
    """Central differences of sum(v * render) with the decisions held fixed
    equal the analytic backward for all 14 parameter kinds of every
    Gaussian (clamped alphas and pixels stopped at T_min included)."""
    cam, p = _dense_scene()
    v = np.random.default_rng(33).uniform(-1, 1, (3, cam.height, cam.width))
    grads, _ = orc.render_backward(p, cam, v, CFG)
    fl = orc.FrozenLists(p, cam, CFG)
    gauss = np.repeat(np.arange(len(p)), len(FD_SLOTS))
    slots = np.tile(FD_SLOTS, len(p))
    fd = fl.fd(p, v, gauss, slots, h=1e-4)
    an = grads[gauss, slots]
    for s in FD_SLOTS:
        m = slots == s
        gmax = np.abs(an[m]).max()
        assert gmax > 0, s
        err = np.abs(fd[m] - an[m])
        assert (err <= 2e-4 * np.maximum(np.abs(an[m]), 1e-3 * gmax) + 1e-10).all(), (s, err.max(), gmax)


def test_gradient_term_magnitudes(orc):
    """render_backward_terms: the same gradient as render_backward; per
    Gaussian, the absolute sums bound the 2D gradient (triangle inequality)
    and equal it where one term contributes; the term counts are the
    composited pairs of the frozen per-pixel lists."""
    p = synth.gaussians(300, 41)
    cam = synth.orbit_camera(40, 32, 25.0)
    dl = np.random.default_rng(3).uniform(-1, 1, (3, 32, 40))
    g_ref, g2_ref = orc.render_backward(p, cam, dl, CFG)
    g, g2, a2, nterm = orc.render_backward_terms(p, cam, dl, CFG)
    # the FP64 sums take their terms in the order the threads reach them
    np.testing.assert_allclose(g, g_ref, rtol=1e-11, atol=1e-13 * np.abs(g_ref).max())
    np.testing.assert_allclose(g2, g2_ref, rtol=1e-11, atol=1e-13 * np.abs(g2_ref).max())
    assert np.all(a2 >= np.abs(g2) * (1 - 1e-12))
    lists = orc.FrozenLists(p, cam, CFG)
    counts = np.bincount(lists.g[:lists.offsets[-1]], minlength=len(p))
    np.testing.assert_array_equal(nterm, counts)
    # one pixel: every Gaussian contributes one term, so the sums are exact
    _, g21, a21, n1 = orc.render_backward_terms(p, cam, dl[:, 16:17, 20:21], CFG, window=(20, 16, 1, 1))
    one = n1 == 1
    assert one.sum() > 3 and n1.max() == 1
    np.testing.assert_allclose(a21[one], np.abs(g21[one]), rtol=1e-12, atol=0)
    # |J a| <= |J| |a| for the packed gradient
    bound = orc.grad_abs_map(p, cam, a2, CFG)
    assert np.all(np.abs(g) <= bound * (1 + 1e-9) + 1e-300)
    assert np.all(bound[nterm == 0] == 0.0)


def test_grad_abs_map_closed_form_columns(orc):
    """Columns of the 2D-record-to-parameter Jacobian whose form is plain:
    dL/dmx reaches the mean through the pinhole projection only
    (d mx / d t = (fx / tz, 0, -fx tx / tz^2), camera rotation identity), the
    opacity-logit record reaches slot 3 alone, and the colour records reach
    the colour slots one to one."""
    cam = _axis_cam()
    p = _one([0.8, 0.3, 1.2], [math.log(0.06)] * 3, [0.9, 0.1, -0.2, 0.3], 0.2, [0.4, 0.5, 0.6])
    tx, tz = float(p[0, 0]) - 0.5, float(p[0, 2]) + 1.0
    assert np.allclose(np.asarray(cam.R, np.float64), np.eye(3))
    for k, want in [(0, {0: cam.fx / tz, 2: cam.fx * abs(tx) / tz ** 2}), (5, {3: 1.0}),
                    (6, {12: 1.0}), (7, {13: 1.0}), (8, {14: 1.0})]:
        m = np.zeros((1, 9))
        m[0, k] = 2.0
        out = orc.grad_abs_map(p, cam, m, CFG)[0]
        expect = np.zeros(16)
        for j, v in want.items():
            expect[j] = 2.0 * v
        np.testing.assert_allclose(out, expect, rtol=1e-9, atol=1e-12)


def test_leaves_are_the_render_where_nothing_is_marginal(orc):
    """render_leaves: one leaf, render's value bit for bit, on every pixel the
    render does not flag; on a flagged pixel more than one leaf, render's
    value among them."""
    p = synth.gaussians(1024, synth.BASE_SEED + 2)
    cam = synth.orbit_camera(96, 80, 30.0)
    img, marg, _, _ = orc.render(p, cam, CFG)
    lv, n = orc.render_leaves(p, cam, CFG)
    assert n.min() >= 1 and marg.sum() > 5
    np.testing.assert_array_equal(marg, n > 1)
    one = n == 1
    np.testing.assert_array_equal(lv[one][:, 0, :].T, img[:, one])
    d = np.abs(lv - img.transpose(1, 2, 0)[:, :, None, :]).max(-1)
    d = np.where(np.arange(lv.shape[2])[None, None, :] < n[:, :, None], d, np.inf).min(-1)
    assert d.max() == 0.0


def _centre_pixel_gaussians(alphas, rgbs, cam):
    """Gaussians on the optical axis in depth order, each with peak alpha
    sigmoid(logit) at the centre pixel (the FP32 logit of the given alpha)."""
    p = np.concatenate([_one([0.5, 0.5, 0.4 + 0.1 * k], [math.log(0.05)] * 3, [1, 0, 0, 0],
                             math.log(a / (1 - a)), rgb) for k, (a, rgb) in enumerate(zip(alphas, rgbs))])
    return p, [1 / (1 + math.exp(-float(x))) for x in p[:, 3]]


def test_leaves_of_a_marginal_alpha_min_decision(orc):
    """A Gaussian whose alpha at the pixel centre lies within the margin
    above 1/255: the pixel may composite it (c alpha) or drop it (0)."""
    cam = _axis_cam()
    p, (a,) = _centre_pixel_gaussians([(1 / 255) * (1 + 5e-5)], [(0.8, 0.4, 0.2)], cam)
    lv, n = orc.render_leaves(p, cam, CFG, window=(32, 32, 1, 1))
    assert n[0, 0] == 2
    got = sorted(tuple(lv[0, 0, k]) for k in range(2))
    np.testing.assert_allclose(got[0], [0, 0, 0], atol=0)
    np.testing.assert_allclose(got[1], p[0, 12:15].astype(np.float64) * a, rtol=1e-12)
    # and its colour gradient lies between the two: 0 (dropped) and alpha (taken)
    lo, hi, _, nterm, nl = orc.render_backward_bounds(p, cam, np.ones((3, 1, 1)), CFG, window=(32, 32, 1, 1))
    assert nl[0, 0] == 2 and nterm[0] == 1
    np.testing.assert_allclose(lo[0, 6:9], 0.0, atol=0)
    np.testing.assert_allclose(hi[0, 6:9], a, rtol=1e-12)


def test_leaves_of_a_marginal_t_min_stop(orc):
    """Two Gaussians on the axis whose transmittance after the second lands
    within the margin above T_min: the pixel may composite the second (FP64
    does) or stop before it."""
    cam = _axis_cam()
    a1 = 0.99
    a2 = 1 - 1e-4 * (1 + 5e-5) / (1 - a1)
    (p, (b1, b2)) = _centre_pixel_gaussians([a1, a2], [(1.0, 0.5, 0.25), (0.2, 0.6, 1.0)], cam)
    cfg = dict(CFG, alpha_max=0.999)
    lv, n = orc.render_leaves(p, cam, cfg, window=(32, 32, 1, 1))
    # T after both: (1 - b1)(1 - b2), b2 as the FP32 logit gives it
    t2 = (1 - b1) * (1 - b2)
    assert abs(t2 / 1e-4 - 1) < 2e-4, t2
    assert n[0, 0] == 2
    first = p[0, 12:15].astype(np.float64) * b1
    both = first + p[1, 12:15].astype(np.float64) * b2 * (1 - b1)
    got = sorted((tuple(lv[0, 0, k]) for k in range(2)), key=lambda v: v[2])
    np.testing.assert_allclose(got[0], first, rtol=1e-12)
    np.testing.assert_allclose(got[1], both, rtol=1e-12)


def test_backward_bounds_and_projection_match_the_backward(orc):
    """Without marginal decisions the bounds collapse to the backward's 2D
    record, and project_backward of that record is the backward's packed
    gradient; with them, the record lies inside the bounds."""
    p = synth.gaussians(600, 44)
    cam = synth.orbit_camera(48, 40, 35.0)
    dl = np.random.default_rng(4).uniform(-1, 1, (3, 40, 48))
    _, marg, _, _ = orc.render(p, cam, CFG, grad_margins=True)
    g, g2 = orc.render_backward(p, cam, dl, CFG)
    lo, hi, ab, nterm, nl = orc.render_backward_bounds(p, cam, dl, CFG)
    assert nl.min() >= 1 and marg.sum() > 0
    np.testing.assert_array_equal(marg, nl > 1)
    scale = np.abs(g2).max()
    assert np.all(lo <= g2 + 1e-12 * scale) and np.all(g2 <= hi + 1e-12 * scale)
    dz = dl.copy()
    dz[:, marg] = 0.0
    g_z, g2_z = orc.render_backward(p, cam, dz, CFG)
    lo_z, hi_z, _, _, _ = orc.render_backward_bounds(p, cam, dz, CFG)
    np.testing.assert_allclose(lo_z, g2_z, rtol=1e-11, atol=1e-13 * scale)
    np.testing.assert_allclose(hi_z, g2_z, rtol=1e-11, atol=1e-13 * scale)
    np.testing.assert_allclose(orc.project_backward(p, cam, g2_z, CFG), g_z, rtol=1e-11,
                               atol=1e-13 * np.abs(g_z).max())
