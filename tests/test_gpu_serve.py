"""Continuous-batching server: every view request's images are the same
whether it was rendered alone or in a batch with other requests while another
scene retrains; the retrained cache matches the same retraining done alone;
a tight HBM budget still serves every request (one per batch); the plain
one-view-per-call path serves the same trace with the same images."""
import copy

import numpy as np
import pytest

from paper_2507_19718_gb300 import synth

pytestmark = pytest.mark.gpu

RES = ((64, 48), (96, 64), (40, 40))


def _scenes(serve, n=3):
    out = []
    for k in range(n):
        pos, rgba = synth.transfer_function(4, 50 + k)
        sc = synth.Scene(density=synth.blob_volume(24, 4, 60 + k), tf_pos=pos, tf_rgba=rgba,
                         light_dir=synth.unit([1, 1, 1]), light_radiance=np.full(3, 3.0, np.float32),
                         env_radiance=np.full(3, 0.3, np.float32))
        out.append(serve.ResidentScene(sc, synth.level_sizes(1500 + 500 * k, 2), seed=700 + 10 * k))
    return out


def _trace(serve):
    # a burst: requests queue up while earlier ones are on the GPU
    tr = serve.poisson_trace(20000.0, 0.004, 3, seed=5, tf_fraction=0.0, resolutions=RES)
    tr = [r for r in tr if r.scene != 2]
    tr.append(serve.Request(len(tr) + 1000, "tf", 2, 0.0005, tf_seed=77))
    for i, r in enumerate(sorted(tr, key=lambda r: r.arrival)):
        r.rid = i
    return tr


def _alone(gsc, sc, r, cfg, ws):
    cam = gsc.camera(synth.orbit_camera(r.width, r.height, r.angle))
    return [gsc.cache_render(L.params, cam, cfg, ws).clone() for L in sc.levels]


def test_batched_results_equal_alone_and_retraining_matches(gpu):
    import torch
    from paper_2507_19718_gb300 import serve
    cfg = gpu.raster_cfg(tile=(16, 16), list_capacity=256, bin_size=32, pixels_per_thread=2)
    scenes = _scenes(serve)
    twin = _scenes(serve)[2]  # same initial cache and volume as scene 2
    srv = serve.Server(scenes, cfg, max_views=8, train_res=(48, 40), retrain_frames=6, max_res=(96, 64),
                       keep_images=True)
    trace = _trace(serve)
    srv.run_batched(trace)
    assert all(r.done == r.done for r in trace)
    views = [r for r in trace if r.kind == "view"]
    assert len(views) > 40
    assert srv.stats["mean_views_per_batch"] > 2  # requests were batched
    ws = gpu.Workspace(4000, 1 << 20, 96, 64)
    for r in views:
        for got, ref in zip(r.images, _alone(gpu, scenes[r.scene], r, cfg, ws)):
            assert torch.equal(got, ref), r.rid
    # the retraining of scene 2 in the mix equals the same retraining alone
    assert scenes[2].frames_trained == 6
    twin.set_tf(77)
    trainer = serve.Trainer(48, 40, 2, 4000, cfg)
    twin.static_frames = 0  # the TF change resets the Eq. 4 schedule
    for f in range(6):
        trainer.frame(twin, angle=30.0, frame=f, seed=srv.seed + 2000)
    torch.cuda.synchronize()
    for k, (La, Lb) in enumerate(zip(scenes[2].levels, twin.levels)):
        a, b = La.params.cpu().numpy(), Lb.params.cpu().numpy()
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-5)
        assert not np.array_equal(a, synth.gaussians(La.n, 720 + k))  # it did train


def test_tight_budget_admits_one_request_at_a_time(gpu):
    from paper_2507_19718_gb300 import serve
    cfg = gpu.raster_cfg()
    scenes = _scenes(serve)
    srv = serve.Server(scenes, cfg, max_views=8, train_res=(48, 40), retrain_frames=2, max_res=(96, 64))
    smallest = min(3 * w * h * 4 * 2 for w, h in RES)
    srv.budget = srv.fixed_bytes + smallest  # two requests never fit together
    trace = [r for r in _trace(serve) if r.kind == "view"][:30]
    srv.run_batched(trace)
    assert all(r.done == r.done for r in trace)
    assert srv.stats["mean_views_per_batch"] == pytest.approx(2.0)


def test_plain_path_serves_the_same_images(gpu):
    import torch
    from paper_2507_19718_gb300 import serve
    cfg = gpu.raster_cfg()
    scenes = _scenes(serve)
    srv = serve.Server(scenes, cfg, max_views=8, train_res=(48, 40), retrain_frames=2, max_res=(96, 64),
                       keep_images=True)
    trace = [r for r in _trace(serve) if r.kind == "view"][:40]
    srv.run_plain(copy.deepcopy(trace))
    plain = srv.run_plain(trace)
    lat = serve.latency_stats(plain)
    assert lat["n"] == 40 and lat["p99_ms"] >= lat["p50_ms"] > 0
    ws = gpu.Workspace(4000, 1 << 20, 96, 64)
    for r in plain:
        for got, ref in zip(r.images, _alone(gpu, scenes[r.scene], r, cfg, ws)):
            assert torch.equal(got, ref)


def test_per_resolution_view_launches_serve_the_same_images(gpu):
    """tune_views picks each request resolution's launch configuration; the
    batched and the plain paths then render with it, and every image is the
    same bits as the default configuration alone (results do not depend on
    tile, bin, staging or pixels per thread)."""
    import torch
    from paper_2507_19718_gb300 import serve
    cfg = gpu.raster_cfg()
    scenes = _scenes(serve)
    srv = serve.Server(scenes, cfg, max_views=8, train_res=(48, 40), retrain_frames=2, max_res=(96, 64),
                       keep_images=True)
    from paper_2507_19718_gb300 import autotune
    space = dict(tiles=((16, 16), (8, 8)), bins=(0,), caps=(128, 256), ppts=(1, 2))
    trials = srv.tune_views(scenes[2], resolutions=RES, **space)
    n = len(list(autotune.candidates(**space)))
    assert n >= 3 and set(trials) == set(RES) and all(len(t) == n for t in trials.values())
    assert set(srv.view_cfgs) == set(RES)
    trace = [r for r in _trace(serve) if r.kind == "view"][:30]
    batched = srv.run_batched(copy.deepcopy(trace))
    plain = srv.run_plain(copy.deepcopy(trace))
    ws = gpu.Workspace(4000, 1 << 20, 96, 64)
    for rb, rp in zip(batched, plain):
        ref = _alone(gpu, scenes[rb.scene], rb, cfg, ws)
        for got_b, got_p, want in zip(rb.images, rp.images, ref):
            assert torch.equal(got_b, want) and torch.equal(got_p, want), rb.rid
