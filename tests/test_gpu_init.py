"""GPU cache initialisation (gsc_cache_init, Sec. 3.2 and Eq. 3) against the
oracle: the delta-tracked points bit for bit (the sampling runs the tracer's
FP32 arithmetic, compared with the oracle's FP32 mirror), the 3-NN distances
and Eq. 3 scales to FP32 rounding, at 4,096 points in full and at the
paper's 300k points on samples."""
import numpy as np
import pytest

from paper_2507_19718_gb300 import synth

pytestmark = pytest.mark.gpu


def _scene(gsc, sc):
    return gsc.Scene.from_synth(sc, "cuda")


def test_init_matches_oracle_small(gpu, orc):
    sc = synth.scene_tiny()
    params, levels = gpu.cache_init(_scene(gpu, sc), 4096, 3, seed=13)
    ref = orc.init_gaussians(sc, 4096, 3, seed=13)
    for got, want in zip(levels, ref):
        got = got.cpu().numpy().astype(np.float64)
        np.testing.assert_array_equal(got[:, 0:3], want[:, 0:3])        # positions: bit for bit
        np.testing.assert_array_equal(got[:, 12:15], want[:, 12:15].astype(np.float32))
        np.testing.assert_allclose(got[:, 3], want[:, 3], atol=1e-6)
        np.testing.assert_array_equal(got[:, 8:12], want[:, 8:12])
        assert not got[:, [7, 15]].any()
        np.testing.assert_allclose(got[:, 4:7], want[:, 4:7], atol=2e-5)


def test_init_full_size_sampled(gpu, orc):
    spatial = pytest.importorskip("scipy.spatial")
    sc = synth.scene_frame(256, seed=synth.BASE_SEED + 1)
    N, K = 300_000, 3
    params, levels = gpu.cache_init(_scene(gpu, sc), N, K, seed=41)
    lv = [L.cpu().numpy().astype(np.float64) for L in levels]
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(N, 500, replace=False))
    pos, alb, att = orc.init_points(sc, N, seed=41, idx=idx)
    assert (att > 0).all()
    np.testing.assert_array_equal(lv[0][idx, 0:3], pos)
    np.testing.assert_array_equal(lv[0][idx, 12:15], alb.astype(np.float32))
    for k, L in enumerate(lv):
        pts = L[:, 0:3]
        np.testing.assert_array_equal(pts, lv[0][:len(L), 0:3])  # level k = the first N >> k points
        d, _ = spatial.cKDTree(pts).query(pts, k=4)
        mbar = d[:, 1:].mean(1)
        q = rng.choice(len(L), 200, replace=False)
        np.testing.assert_allclose(orc.knn3_mean(pts, q), mbar[q], rtol=1e-12)   # the library query is exact
        s, mu, sigma = orc.init_scales(mbar)
        assert (mbar > mu + 2 * sigma).any()  # the cap is active on real data
        np.testing.assert_allclose(L[:, 4], np.log(s), atol=5e-5)


def test_init_of_an_empty_volume_reports_the_points_it_could_not_place(gpu):
    sc = synth.scene_tiny()
    sc.tf_rgba = sc.tf_rgba.copy()
    sc.tf_rgba[:, 3] = 0.0  # transparent everywhere: no collision can happen
    with pytest.raises(gpu.GscError) as e:
        gpu.cache_init(_scene(gpu, sc), 64, 1, seed=1, max_attempts=16)
    assert e.value.status == gpu.GSC_ERR_TIMEOUT
