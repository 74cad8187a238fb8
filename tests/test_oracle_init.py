"""Pins of the oracle's cache initialisation (Sec. 3.2 "Cache
Initialization", Eq. 3): delta-tracked point sampling, the 3-NN distances and
the capped isotropic scales.

Sampling is pinned by invariants (points inside the box, only where sigma_t
> 0), a closed form (constant transfer function: albedo = albedo * RGB) and
Beer-Lambert (the mean number of rays per point equals 1 / E[1 - exp(-sigma
l)] over the ray distribution, estimated independently); the 3-NN distances
by a k-d tree library query; Eq. 3 by lattices whose distances are known.
"""
import numpy as np
import pytest

from paper_2507_19718_gb300 import synth


def _homogeneous(sigma, rgb=(0.2, 0.5, 0.9)):
    pos = np.array([0.0, 1.0], np.float32)
    rgba = np.array([[*rgb, 1.0], [*rgb, 1.0]], np.float32)
    sc = synth.Scene(density=np.full((8, 8, 8), 1.0, np.float32), tf_pos=pos, tf_rgba=rgba,
                     light_dir=synth.unit([0, 0, 1]), light_radiance=np.zeros(3, np.float32),
                     env_radiance=np.zeros(3, np.float32))
    sc.density_max = 1.0
    sc.sigma_max = float(sigma)
    return sc


def test_points_lie_in_the_box_where_sigma_t_is_positive(orc):
    sc = synth.scene_tiny()
    pos, alb, att = orc.init_points(sc, 4000, seed=3)
    assert (att > 0).all()
    assert (pos >= 0).all() and (pos <= 1).all()
    assert (orc.sigma_t(sc, pos) > 0).all()
    # the FP32 mirror and FP64 sample the same distribution
    p64, _, a64 = orc.init_points(sc, 4000, seed=3, precision=64)
    assert np.abs(p64.mean(0) - pos.mean(0)).max() < 0.02
    assert abs(a64.mean() - att.mean()) < 0.2 * att.mean()


def test_constant_transfer_function_gives_the_albedo_closed_form(orc):
    sc = _homogeneous(5.0)
    _, alb, att = orc.init_points(sc, 500, seed=1, precision=64)
    assert (att > 0).all()
    # the scene stores FP32 values; the product is formed in FP64
    want = np.float64(np.float32(sc.albedo)) * np.array([0.2, 0.5, 0.9], np.float32).astype(np.float64)
    np.testing.assert_allclose(alb, np.tile(want, (500, 1)), rtol=1e-15)


@pytest.mark.parametrize("sigma", [0.7, 2.5])
def test_rays_per_point_follow_beer_lambert(orc, sigma):
    """A ray of chord length l through a homogeneous box collides with
    probability 1 - exp(-sigma l), so rays per point are geometric with mean
    1 / E[1 - exp(-sigma l)].  The expectation is estimated here by a
    separate Monte Carlo of the ray distribution (origin on the unit sphere
    around the box centre, aimed at a uniform point of the box)."""
    sc = _homogeneous(sigma)
    n = 20000
    _, _, att = orc.init_points(sc, n, seed=11, precision=64)
    rng = np.random.default_rng(5)
    m = 400000
    z = rng.uniform(-1, 1, m)
    phi = rng.uniform(0, 2 * np.pi, m)
    r = np.sqrt(1 - z * z)
    o = 0.5 + np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)
    d = rng.uniform(0, 1, (m, 3)) - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    with np.errstate(divide="ignore"):
        t0 = (0 - o) / d
        t1 = (1 - o) / d
    lo = np.minimum(t0, t1).max(1)
    hi = np.maximum(t0, t1).min(1)
    chord = np.maximum(hi - lo, 0)
    p_hit = (1 - np.exp(-sigma * chord)).mean()
    mean_att = att.mean()
    se = np.sqrt((1 - p_hit) / p_hit ** 2 / n)
    assert abs(mean_att - 1 / p_hit) < 5 * se + 1e-3, (mean_att, 1 / p_hit, se)


def test_knn3_mean_matches_a_kdtree(orc):
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(2)
    pts = np.concatenate([rng.uniform(0, 1, (1500, 3)), rng.normal(0.5, 0.01, (500, 3))])
    pts[7] = pts[8]  # a duplicate: distance 0
    got = orc.knn3_mean(pts)
    d, _ = spatial.cKDTree(pts).query(pts, k=4)
    np.testing.assert_allclose(got, d[:, 1:].mean(1), rtol=1e-12, atol=1e-15)
    q = np.array([3, 7, 1999])
    np.testing.assert_allclose(orc.knn3_mean(pts, q), got[q], rtol=0, atol=0)


def test_eq3_on_a_lattice_is_half_the_spacing(orc):
    h = 0.05
    g = np.arange(8) * h
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    mbar = orc.knn3_mean(pts)
    np.testing.assert_allclose(mbar, h, rtol=1e-12)
    s, mu, sigma = orc.init_scales(mbar)
    np.testing.assert_allclose(s, h / 2, rtol=1e-12)
    assert abs(mu - h) < 1e-12 and sigma < 1e-12


def test_eq3_caps_an_outlier_at_two_standard_deviations(orc):
    """A lattice plus one far point: the far point's mean 3-NN distance D is
    the largest, and the cap mu + 2 sigma (over all M points) replaces it."""
    h = 0.05
    g = np.arange(6) * h
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    far = np.array([[2.0, 2.0, 2.0]])
    pts = np.concatenate([lat, far])
    mbar = orc.knn3_mean(pts)
    M = len(pts)
    # the far point's nearest lattice points are the corner (0.25, 0.25, 0.25)
    # and the corner's three axis neighbours; their distances written out
    c = np.array([0.25, 0.25, 0.25])
    dd = sorted([np.linalg.norm(far[0] - c), np.linalg.norm(far[0] - (c - [h, 0, 0])),
                 np.linalg.norm(far[0] - (c - [0, h, 0])), np.linalg.norm(far[0] - (c - [0, 0, h]))])
    D = np.mean(dd[:3])
    assert abs(mbar[-1] - D) < 1e-12
    mu = ((M - 1) * h + D) / M
    sigma = np.sqrt(((M - 1) * (h - mu) ** 2 + (D - mu) ** 2) / M)
    s, mu_o, sig_o = orc.init_scales(mbar)
    assert abs(mu_o - mu) < 1e-12 and abs(sig_o - sigma) < 1e-12
    assert D > mu + 2 * sigma
    assert abs(s[-1] - (mu + 2 * sigma) / 2) < 1e-12
    np.testing.assert_allclose(s[:-1], h / 2, rtol=1e-12)


def test_init_gaussians_layout(orc):
    sc = synth.scene_tiny()
    levels = orc.init_gaussians(sc, 1024, 3, seed=9)
    assert [len(p) for p in levels] == [1024, 512, 256]
    pos, alb, _ = orc.init_points(sc, 1024, seed=9)
    for k, p in enumerate(levels):
        n = 1024 >> k
        np.testing.assert_array_equal(p[:, 0:3], pos[:n].astype(np.float32))
        np.testing.assert_array_equal(p[:, 12:15], alb[:n])
        assert np.allclose(p[:, 3], np.log(0.1 / 0.9))
        assert (p[:, 4] == p[:, 5]).all() and (p[:, 5] == p[:, 6]).all()
        assert (p[:, 8] == 1).all() and not p[:, [7, 9, 10, 11, 15]].any()
    # sparser levels get larger Gaussians
    assert np.exp(levels[2][:, 4]).mean() > np.exp(levels[0][:, 4]).mean()
