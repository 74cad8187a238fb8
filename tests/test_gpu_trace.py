"""GPU volume path tracer (Sec. 3.2 - 3.5) against the oracle's FP32 mirror,
bit for bit, through the C ABI: same Philox4x32-10 streams, same operation
order, no contraction, the same own ln / sincos."""
import numpy as np
import pytest

from paper_2507_19718_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(gpu, scene, cam, **kw):
    import torch
    sc = gpu.Scene.from_synth(scene)
    cache = kw.pop("cache", None)
    if cache is not None:
        cache = torch.from_numpy(np.ascontiguousarray(cache, np.float32)).cuda()
    tg, img = gpu.trace(sc, cam, cache=cache, **kw)
    torch.cuda.synchronize()
    return (tg.cpu().numpy() if tg is not None else None), img.cpu().numpy()


def test_trace_bit_exact_config0(gpu, orc):
    scene = synth.scene_tiny()
    cam = synth.orbit_camera(128, 128, 30.0)
    tg, img = _run(gpu, scene, cam, spp=4, max_bounces=4, levels=4, seed=synth.BASE_SEED, frame=3)
    rt, ri = orc.trace(scene, cam, spp=4, max_bounces=4, levels=4, seed=synth.BASE_SEED, frame=3, precision=32)
    assert ri.max() > 0.01 and rt[1].max() > 0
    np.testing.assert_array_equal(img, ri.astype(np.float32))
    np.testing.assert_array_equal(tg, rt.astype(np.float32))


def test_trace_bit_exact_with_cache_and_termination(gpu, orc):
    scene = synth.scene_tiny()
    scene.env_radiance = np.array([0.2, 0.25, 0.3], np.float32)
    cam = synth.orbit_camera(64, 48, 120.0)
    cache = synth.uniform_image(4 * 3, 48, 64, 8).reshape(4, 3, 48, 64)
    kw = dict(spp=2, max_bounces=6, levels=4, seed=77, frame=0, C_term=0.5, eps=1e-6)
    tg, img = _run(gpu, scene, cam, cache=cache, **kw)
    rt, ri = orc.trace(scene, cam, spp=2, max_bounces=6, levels=4, seed=77, frame=0, C=0.5, eps=1e-6,
                       cache=cache, precision=32)
    np.testing.assert_array_equal(img, ri.astype(np.float32))
    np.testing.assert_array_equal(tg, rt.astype(np.float32))


@pytest.mark.parametrize("C", [0.5, 2.0])
def test_trace_bit_exact_with_per_call_tr_out(gpu, orc, C):
    """Algorithm 1 with Tr_out read per call (each call starts from the
    albedo product and divides by its own Tr + eps), bit for bit against the
    FP32 mirror, and different from the cumulative reading.  C = 2 lets some
    calls return Tr >= 0.9 (no roulette, the undivided product)."""
    scene = synth.scene_tiny()
    scene.env_radiance = np.array([0.2, 0.25, 0.3], np.float32)
    cam = synth.orbit_camera(64, 48, 120.0)
    cache = synth.uniform_image(4 * 3, 48, 64, 8).reshape(4, 3, 48, 64)
    kw = dict(spp=2, max_bounces=6, levels=4, seed=78, frame=1, C_term=C, eps=1e-6)
    tg, img = _run(gpu, scene, cam, cache=cache, tr_out=gpu.TR_OUT_PER_CALL, **kw)
    rt, ri = orc.trace(scene, cam, spp=2, max_bounces=6, levels=4, seed=78, frame=1, C=C, eps=1e-6,
                       cache=cache, precision=32, tr_out=1)
    np.testing.assert_array_equal(img, ri.astype(np.float32))
    np.testing.assert_array_equal(tg, rt.astype(np.float32))
    tc, _ = _run(gpu, scene, cam, cache=cache, tr_out=gpu.TR_OUT_CUMULATIVE, **kw)
    assert not np.array_equal(tc, tg)


def test_trace_bit_exact_frame_scene_1080p_windows(gpu, orc):
    """The 1080p frame workload (256^3 blobs + fBm, 8-point TF, directional +
    environment light, 1 spp, 8 bounces, 3 levels) on sampled windows.  A frame
    of this size runs the many-wave register budget of the tracer (16 CTAs per
    SM); the small frames of the other tests run the spill-free one."""
    scene = synth.scene_frame()
    cam = synth.orbit_camera(1920, 1080, 45.0)
    tg, img = _run(gpu, scene, cam, spp=1, max_bounces=8, levels=3, seed=5, frame=11)
    for (x0, y0) in [(950, 530), (600, 700), (1500, 200), (0, 0), (1904, 1072)]:
        win = (x0, y0, 16, 8)
        rt, ri = orc.trace(scene, cam, spp=1, max_bounces=8, levels=3, seed=5, frame=11, window=win,
                           precision=32)
        np.testing.assert_array_equal(img[:, y0:y0 + 8, x0:x0 + 16], ri.astype(np.float32))
        np.testing.assert_array_equal(tg[:, :, y0:y0 + 8, x0:x0 + 16], rt.astype(np.float32))
    assert img.max() > 0


def test_tf_change_changes_image(gpu):
    import torch
    scene = synth.scene_tiny()
    cam = synth.orbit_camera(48, 48, 10.0)
    sc = gpu.Scene.from_synth(scene)
    _, a = gpu.trace(sc, cam, spp=1, max_bounces=3, levels=2, seed=1)
    a = a.clone()
    pos, rgba = synth.transfer_function(8, 999)
    sc.set_tf(pos, rgba)
    _, b = gpu.trace(sc, cam, spp=1, max_bounces=3, levels=2, seed=1)
    torch.cuda.synchronize()
    assert not torch.equal(a, b)


def test_trace_bit_exact_with_two_sphere_lights(gpu, orc):
    """The paper's two-point lighting (two spherical area lights outside the
    volume, Sec. 4.3) with the environment on, 4 spp, bit for bit."""
    scene = synth.scene_tiny()
    scene.light_radiance = np.zeros(3, np.float32)
    scene.env_radiance = np.array([0.1, 0.1, 0.12], np.float32)
    scene.spheres = synth.two_sphere_lights()
    cam = synth.orbit_camera(96, 72, 200.0)
    tg, img = _run(gpu, scene, cam, spp=4, max_bounces=5, levels=3, seed=5, frame=2)
    rt, ri = orc.trace(scene, cam, spp=4, max_bounces=5, levels=3, seed=5, frame=2, precision=32)
    assert ri.max() > 0.01
    np.testing.assert_array_equal(img, ri.astype(np.float32))
    np.testing.assert_array_equal(tg, rt.astype(np.float32))


def test_sphere_light_outside_the_box_is_required(gpu):
    scene = synth.scene_tiny()
    scene.spheres = [(np.array([0.5, 0.5, 1.05], np.float32), 0.1, np.ones(3, np.float32))]
    with pytest.raises(gpu.GscError):
        gpu.Scene.from_synth(scene)
