"""Batched rendering (gsc_render_batch): views of uneven resolution across
several scenes in one binning and one persistent launch.  Each view's image is
bit-identical to rendering it alone, each scene's gradient equals the sum of
its views' gradients computed alone (up to the order of FP32 atomics), and
the whole forward + backward replays from a captured CUDA graph."""
import numpy as np
import pytest

from parity import fp32_sum_bar

from paper_2507_19718_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [(64, 48), (100, 75), (128, 128), (37, 29), (96, 80)]


def _setup(gsc):
    import torch
    scenes = [torch.from_numpy(synth.gaussians(n, 300 + k)).cuda() for k, n in enumerate([300, 500, 800])]
    views = []
    for i, (w, h) in enumerate(SIZES):
        cam = gsc.camera(synth.orbit_camera(w, h, 37.0 * i))
        views.append(dict(params=scenes[i % 3], cam=cam, scene=i % 3,
                          image=torch.zeros((3, h, w), device="cuda"),
                          dL_dimage=torch.from_numpy(
                              np.random.default_rng(i).uniform(-1, 1, (3, h, w)).astype(np.float32)).cuda()))
    return scenes, views


def _ws(gsc, scenes, nviews):
    total = sum(int(s.shape[0]) for s in scenes) * 2
    return gsc.Workspace(total, 1 << 22, 128, 128, max_views=nviews)


@pytest.mark.parametrize("tile,ppt", [((16, 16), 2), ((8, 8), 1)])
def test_batch_matches_views_alone(gpu, tile, ppt):
    import torch
    scenes, views = _setup(gpu)
    cfg = gpu.raster_cfg(tile=tile, list_capacity=256, bin_size=32, pixels_per_thread=ppt)
    ws = _ws(gpu, scenes, len(views))
    grads = [torch.zeros_like(s) for s in scenes]
    for v in views:
        v["grads"] = grads[v["scene"]]
    gpu.render_batch(views, gpu.BATCH_FWD | gpu.BATCH_BWD, cfg, ws)
    ws.status()
    alone_ws = gpu.Workspace(max(int(s.shape[0]) for s in scenes), 1 << 22, 128, 128)
    ref_grads = [torch.zeros_like(s) for s in scenes]
    for v in views:
        img = gpu.cache_render(v["params"], v["cam"], cfg, alone_ws)
        gpu.cache_backward(v["params"], v["cam"], cfg, alone_ws, v["dL_dimage"], ref_grads[v["scene"]])
        alone_ws.status()
        assert torch.equal(img, v["image"])
        assert float(img.abs().max()) > 0
    for g, r in zip(grads, ref_grads):
        g, r = g.cpu().numpy(), r.cpu().numpy()
        np.testing.assert_allclose(g, r, rtol=1e-4, atol=1e-6 * np.abs(r).max())
        assert np.abs(r).max() > 0


def test_batch_with_an_empty_view(gpu):
    import torch
    scenes, views = _setup(gpu)
    empty = torch.zeros((0, 16), device="cuda")
    views[1]["params"] = empty
    views[1]["image"].fill_(5.0)
    cfg = gpu.raster_cfg()
    ws = _ws(gpu, scenes, len(views))
    gpu.render_batch(views, gpu.BATCH_FWD, cfg, ws)
    ws.status()
    assert float(views[1]["image"].abs().max()) == 0.0
    alone = gpu.cache_render(views[2]["params"], views[2]["cam"], cfg, ws)
    assert torch.equal(alone, views[2]["image"])


def test_batch_replays_from_a_cuda_graph(gpu):
    import torch
    scenes, views = _setup(gpu)
    cfg = gpu.raster_cfg(tile=(16, 16), list_capacity=256, bin_size=64, pixels_per_thread=2)
    ws = _ws(gpu, scenes, len(views))
    grads = [torch.zeros_like(s) for s in scenes]
    for v in views:
        v["grads"] = grads[v["scene"]]

    def step():
        for g in grads:
            g.zero_()
        gpu.render_batch(views, gpu.BATCH_FWD | gpu.BATCH_BWD, cfg, ws)

    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        step()  # eager warm-up on the capture stream
    torch.cuda.synchronize()
    eager_imgs = [v["image"].clone() for v in views]
    eager_grads = [g.clone() for g in grads]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        step()
    for v in views:
        v["image"].zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    ws.status()
    for v, e in zip(views, eager_imgs):
        assert torch.equal(v["image"], e)
    for g, e in zip(grads, eager_grads):
        np.testing.assert_allclose(g.cpu().numpy(), e.cpu().numpy(), rtol=1e-4,
                                   atol=1e-6 * float(e.abs().max()))


def test_frame_loop_fused_levels_match_per_level_calls(gpu):
    """The frame loop's fused path (all levels in one training step with the
    loss folded in, one AdamW launch over the contiguous store) gives the
    per-level path's renders bit for bit and the same trained parameters (up
    to the order of the FP32 gradient atomics and of the loss sums)."""
    import torch
    from paper_2507_19718_gb300.frame import FrameLoop
    sc = synth.scene_tiny()
    sizes = synth.level_sizes(1200, 3)
    kw = dict(spp=1, max_bounces=3, tile=(16, 16), list_capacity=256, bin_size=32)
    a = FrameLoop(sc, sizes, 96, 72, fused=True, **kw)
    b = FrameLoop(sc, sizes, 96, 72, fused=False, **kw)
    for f in range(3):
        cam = synth.orbit_camera(96, 72, 5.0 * f)
        la = a.frame(cam, f).clone()
        lb = b.frame(cam, f).clone()
        if f == 0:
            assert torch.equal(a.renders, b.renders)
            assert torch.equal(a.targets, b.targets)
            # the fused training step sums the loss per tile: same terms, other order
            np.testing.assert_allclose(la.cpu().numpy(), lb.cpu().numpy(), rtol=2e-6)
    a.ws.status()
    b.ws.status()
    for La, Lb in zip(a.levels, b.levels):
        np.testing.assert_allclose(La.params.cpu().numpy(), Lb.params.cpu().numpy(), rtol=1e-4, atol=1e-5)
    assert float(a.renders.abs().max()) > 0


def test_frame_to_host_matches_frame_then_copies(gpu):
    """FrameLoop.frame_to_host (image copied on a side stream while the levels
    train, on a stream of the caller's) returns what frame() followed by the
    two copies returns: the traced image bit for bit every frame, the losses
    bit for bit on the first frame and to the order of the gradient atomics
    after it."""
    import torch
    from paper_2507_19718_gb300.frame import FrameLoop
    sc = synth.scene_tiny()
    sizes = synth.level_sizes(1200, 3)
    kw = dict(spp=1, max_bounces=3, tile=(16, 16), list_capacity=256, bin_size=32)
    a = FrameLoop(sc, sizes, 96, 72, **kw)
    b = FrameLoop(sc, sizes, 96, 72, **kw)
    hi = torch.empty((3, 72, 96), pin_memory=True)
    hl = torch.empty((3,), pin_memory=True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    for f in range(3):
        cam = synth.orbit_camera(96, 72, 5.0 * f)
        la = a.frame(cam, f).cpu()
        ia = a.image.cpu()
        b.frame_to_host(cam, f, hi, hl, s)
        s.synchronize()
        assert torch.equal(hi, ia)
        if f == 0:
            assert torch.equal(hl, la)
        else:
            np.testing.assert_allclose(hl.numpy(), la.numpy(), rtol=1e-4)
    torch.cuda.synchronize()
    a.ws.status()
    b.ws.status()
    assert float(ia.abs().max()) > 0


def test_frame_loop_adaptive_training_launch(gpu):
    """FrameLoop.adapt_train_launch: every candidate runs (the explored
    frames), every timed step is reported, and the trained cache is the one
    the fixed configuration gives, up to the order of the FP32 sums."""
    import torch
    from paper_2507_19718_gb300.frame import FrameLoop
    sc = synth.scene_tiny()
    sizes = synth.level_sizes(1200, 3)
    kw = dict(spp=1, max_bounces=3, tile=(16, 16), list_capacity=256, bin_size=32)
    a = FrameLoop(sc, sizes, 96, 72, **kw)
    b = FrameLoop(sc, sizes, 96, 72, **kw)
    cfgs = [gpu.raster_cfg(tile=(16, 16), list_capacity=96, bin_size=32, pixels_per_thread=4),
            gpu.raster_cfg(tile=(16, 16), list_capacity=128, bin_size=32, pixels_per_thread=2),
            gpu.raster_cfg(tile=(16, 16), list_capacity=256, bin_size=32, pixels_per_thread=1)]
    sel = a.adapt_train_launch(cfgs, explore_every=2)
    b.cfg_bwd = cfgs[0]
    frames = 6
    for f in range(frames):
        cam = synth.orbit_camera(96, 72, 5.0 * f)
        la = a.frame(cam, f).clone()
        lb = b.frame(cam, f).clone()
        if f == 0:
            np.testing.assert_allclose(la.cpu().numpy(), lb.cpu().numpy(), rtol=2e-6)
    torch.cuda.synchronize()
    a._adapt_collect(lag=0)
    assert sum(sel.runs) == frames and all(r > 0 for r in sel.runs)
    assert all(e is not None and e > 0 for e in sel.est)
    a.ws.status()
    b.ws.status()
    # Adam normalises each step, so a gradient near zero whose sign depends on
    # the summation order moves its parameter by a full step: compare all but
    # a few elements to the tolerance of the fused-level test
    for La, Lb in zip(a.levels, b.levels):
        pa, pb = La.params.cpu().numpy(), Lb.params.cpu().numpy()
        assert np.isfinite(pa).all()
        assert (np.abs(pa - pb) <= 1e-5 + 1e-4 * np.abs(pb)).mean() > 0.999


@pytest.mark.parametrize("kind", [0, 1])
def test_train_batch_equals_render_loss_backward(gpu, orc, kind):
    """gsc_train_batch (render + HDR loss + backward in one launch) against
    the separate calls on the same views: images bit for bit, losses to
    summation order, gradients to the order of their FP32 sums (the two
    launches may split tiles differently, which regroups the sums): within
    twice the FP32 summation bar of each (Gaussian, slot), summed over the
    views that share the scene, plus 1e-4 relative."""
    import torch
    scenes, views = _setup(gpu)
    cfg = gpu.raster_cfg(tile=(16, 16), list_capacity=256, bin_size=32, pixels_per_thread=2)
    ws = _ws(gpu, scenes, len(views))
    rng = np.random.default_rng(77)
    targets = [torch.from_numpy(rng.uniform(0, 1, v["image"].shape).astype(np.float32)).cuda() for v in views]
    grads_a = [torch.zeros_like(s) for s in scenes]
    losses_a = torch.zeros(len(views), device="cuda")
    imgs_a = [torch.zeros_like(v["image"]) for v in views]
    tv = [dict(params=v["params"], cam=v["cam"], target=t, image=im, grads=grads_a[v["scene"]], loss=losses_a[i])
          for i, (v, t, im) in enumerate(zip(views, targets, imgs_a))]
    gpu.train_batch(tv, cfg, ws, kind)
    ws.status()
    # the same step through the separate calls
    grads_b = [torch.zeros_like(s) for s in scenes]
    for v in views:
        v["grads"] = grads_b[v["scene"]]
    gpu.render_batch(views, gpu.BATCH_FWD, cfg, ws)
    losses_b = []
    for v, t in zip(views, targets):
        val, dl = gpu.loss(kind, v["image"], t, ws)
        v["dL_dimage"] = dl
        losses_b.append(float(val))
    gpu.render_batch(views, gpu.BATCH_BWD, cfg, ws)
    ws.status()
    for v, im in zip(views, imgs_a):
        assert torch.equal(v["image"], im)
    np.testing.assert_allclose(losses_a.cpu().numpy(), losses_b, rtol=2e-6)
    bars = [np.zeros(tuple(s.shape)) for s in scenes]
    for i, v in enumerate(views):
        cam = synth.orbit_camera(*SIZES[i], 37.0 * i)  # the view's camera, as _setup made it
        p_np, dl = v["params"].cpu().numpy(), v["dL_dimage"].cpu().numpy()
        _, _, ab, nterm, _ = orc.render_backward_bounds(p_np, cam, dl)
        bars[v["scene"]] += fp32_sum_bar(orc, p_np, cam, ab, nterm)
    for a, b, bar in zip(grads_a, grads_b, bars):
        a, b = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
        bad = np.abs(a - b) > 2 * bar + 1e-4 * np.abs(b)
        assert not bad.any(), (np.argwhere(bad)[:5].tolist(), a[bad][:5], b[bad][:5], bar[bad][:5])
        assert np.abs(b).max() > 0


def test_train_batch_rejects_non_local_losses(gpu):
    import torch
    scenes, views = _setup(gpu)
    ws = _ws(gpu, scenes, 1)
    v = views[0]
    tv = [dict(params=v["params"], cam=v["cam"], target=torch.zeros_like(v["image"]),
               grads=torch.zeros_like(v["params"]), loss=torch.zeros((), device="cuda"))]
    with pytest.raises(gpu.GscError):
        gpu.train_batch(tv, gpu.raster_cfg(), ws, gpu.LOSS_L1_SSIM)


def test_batched_step_graph_replays_the_training_step(gpu):
    """BatchedStep (one training-step launch for all views under a CUDA graph)
    gives the same losses and gradients as its separate-launch step."""
    import torch
    from paper_2507_19718_gb300 import batched
    scenes = [torch.from_numpy(synth.gaussians(n, 900 + k)).cuda() for k, n in enumerate([400, 700])]
    views = [(k % 2, synth.orbit_camera(w, h, 20.0 * k)) for k, (w, h) in enumerate(SIZES)]
    cfg = gpu.raster_cfg(tile=(16, 16), list_capacity=256, bin_size=32, pixels_per_thread=2)
    st = batched.BatchedStep(scenes, views, cfg, max_pairs=1 << 22)
    st.step_separate()
    torch.cuda.synchronize()
    sep_g = [g.clone() for g in st.grads]
    sep_l = st.losses.clone()
    st.capture()
    st.replay()
    torch.cuda.synchronize()
    st.ws.status()
    np.testing.assert_allclose(st.losses.cpu().numpy(), sep_l.cpu().numpy(), rtol=2e-6)
    for a, b in zip(st.grads, sep_g):
        np.testing.assert_allclose(a.cpu().numpy(), b.cpu().numpy(), rtol=1e-4,
                                   atol=1e-6 * float(b.abs().max()))
        assert float(b.abs().max()) > 0


def test_batch_with_many_bins_matches_views_alone(gpu):
    """Six 1280x720 views with 32-pixel bins: 5,520 bins, so the pair sort
    takes two radix passes (the bin ranges come from the sorted keys) and
    the tile order handles thousands of bins; every image is still the
    single-view render bit for bit."""
    import torch
    scenes = [torch.from_numpy(synth.gaussians(n, 700 + k)).cuda() for k, n in enumerate([1500, 2500])]
    views = []
    for i in range(6):
        cam = gpu.camera(synth.orbit_camera(1280, 720, 23.0 * i))
        views.append(dict(params=scenes[i % 2], cam=cam, scene=i % 2,
                          image=torch.zeros((3, 720, 1280), device="cuda"),
                          dL_dimage=torch.from_numpy(
                              np.random.default_rng(40 + i).uniform(-1, 1, (3, 720, 1280)).astype(np.float32)).cuda()))
    cfg = gpu.raster_cfg(tile=(8, 8), list_capacity=256, bin_size=32, pixels_per_thread=1)
    ws = gpu.Workspace(4000 * 6, 1 << 23, 1280, 720, max_views=6)
    grads = [torch.zeros_like(s) for s in scenes]
    for v in views:
        v["grads"] = grads[v["scene"]]
    gpu.render_batch(views, gpu.BATCH_FWD | gpu.BATCH_BWD, cfg, ws)
    ws.status()
    alone_ws = gpu.Workspace(2500, 1 << 23, 1280, 720)
    ref_grads = [torch.zeros_like(s) for s in scenes]
    for v in views:
        img = gpu.cache_render(v["params"], v["cam"], cfg, alone_ws)
        gpu.cache_backward(v["params"], v["cam"], cfg, alone_ws, v["dL_dimage"], ref_grads[v["scene"]])
        alone_ws.status()
        assert torch.equal(img, v["image"])
        assert float(img.abs().max()) > 0
    # a Gaussian near the camera sums 10^5 pixel terms of random sign per
    # view (three views per scene): the FP32 atomics of the batch and of the
    # single views add them in different orders, which moves such a sum by up
    # to a few 1e-4 of itself
    for g, r in zip(grads, ref_grads):
        g, r = g.cpu().numpy(), r.cpu().numpy()
        np.testing.assert_allclose(g, r, rtol=2e-3, atol=1e-5 * np.abs(r).max())
        assert np.abs(r).max() > 0


def test_train_step_equals_train_batch_then_cache_step(gpu):
    """gsc_train_step (the AdamW step fused into the per-Gaussian gradient
    kernel) against gsc_train_batch followed by gsc_cache_step per level, on
    three levels with gradients already accumulated and moments from earlier
    steps: images bit for bit, losses to summation order, parameters and
    moments to the order of the gradient atomics; Gaussians no tile saw
    (behind the camera) take exactly the step of their accumulated
    gradient."""
    import torch
    rng = np.random.default_rng(91)
    cam = synth.orbit_camera(96, 80, 25.0)
    fwd = cam.R[2].astype(np.float64)
    levels = []
    for k, n in enumerate([700, 350, 175]):
        p = synth.gaussians(n, 900 + k)
        p[:5, 0:3] = (cam.pos - 0.5 * fwd).astype(np.float32)  # behind the camera: never seen
        g = rng.normal(0, 1e-3, (n, 16)).astype(np.float32)
        m = rng.normal(0, 1e-3, (n, 16)).astype(np.float32)
        v = rng.uniform(1e-6, 1e-5, (n, 16)).astype(np.float32)
        levels.append((p, g, m, v))
    target = torch.from_numpy(rng.uniform(0, 1, (3, 80, 96)).astype(np.float32)).cuda()
    cfg = gpu.raster_cfg(tile=(16, 16), list_capacity=256, bin_size=32, pixels_per_thread=4)
    ws = gpu.Workspace(1225, 1 << 22, 96, 80, max_views=3)
    adam = gpu.adam_params(gpu.PAPER_LR, lr_scale=0.7, step=6)

    def state():
        return [tuple(torch.from_numpy(a.copy()).cuda() for a in L) for L in levels]

    def views(st, losses, imgs):
        return [dict(params=P, cam=cam, target=target, image=imgs[k], grads=G, loss=losses[k], m=M, v=V)
                for k, (P, G, M, V) in enumerate(st)]

    sa, la, ia = state(), torch.zeros(3, device="cuda"), [torch.zeros(3, 80, 96, device="cuda") for _ in range(3)]
    gpu.train_batch(views(sa, la, ia), cfg, ws, gpu.LOSS_HDR)
    for P, G, M, V in sa:
        gpu.cache_step(P, G, M, V, adam)
    ws.status()
    sb, lb, ib = state(), torch.zeros(3, device="cuda"), [torch.zeros(3, 80, 96, device="cuda") for _ in range(3)]
    gpu.train_step(views(sb, lb, ib), adam, cfg, ws, gpu.LOSS_HDR)
    ws.status()
    for a, b in zip(ia, ib):
        assert torch.equal(a, b)
    np.testing.assert_allclose(la.cpu().numpy(), lb.cpu().numpy(), rtol=2e-6)
    for (Pa, Ga, Ma, Va), (Pb, Gb, Mb, Vb), (p0, _, _, _) in zip(sa, sb, levels):
        Pa, Ma, Va, Pb, Mb, Vb = (x.cpu().numpy().astype(np.float64) for x in (Pa, Ma, Va, Pb, Mb, Vb))
        assert float(Gb.abs().max()) == 0.0 and float(Ga.abs().max()) == 0.0
        dp = np.abs(Pa - p0)
        assert dp.max() > 0
        assert np.all(np.abs(Pb - Pa) <= 1e-6 * np.abs(Pa) + 1e-3 * dp + 1e-9)
        np.testing.assert_allclose(Mb, Ma, rtol=1e-4, atol=1e-6 * np.abs(Ma).max())
        np.testing.assert_allclose(Vb, Va, rtol=1e-4, atol=1e-6 * np.abs(Va).max())
        # the unseen Gaussians: the same arithmetic on the same gradient
        np.testing.assert_array_equal(Pb[:5], Pa[:5])
        np.testing.assert_array_equal(Mb[:5], Ma[:5])
        np.testing.assert_array_equal(Vb[:5], Va[:5])


def test_train_step_rejects_shared_parameters(gpu):
    import torch
    p = torch.from_numpy(synth.gaussians(100, 5)).cuda()
    g, m, v = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    cam = synth.orbit_camera(32, 32, 0.0)
    t = torch.zeros(3, 32, 32, device="cuda")
    loss = torch.zeros(2, device="cuda")
    ws = gpu.Workspace(200, 1 << 20, 32, 32, max_views=2)
    views = [dict(params=p, cam=cam, target=t, grads=g, loss=loss[k], m=m, v=v) for k in range(2)]
    with pytest.raises(gpu.GscError) as e:
        gpu.train_step(views, gpu.adam_params(gpu.PAPER_LR), gpu.raster_cfg(), ws, gpu.LOSS_HDR)
    assert e.value.status == gpu.GSC_ERR_INVALID_ARG


def test_train_step_without_accumulated_gradient(gpu):
    """grads = None in gsc_train_step means no accumulated gradient: the
    same step as passing zeros (to the order of the gradient atomics;
    Gaussians no tile saw bit for bit)."""
    import torch
    cam = synth.orbit_camera(64, 48, 10.0)
    p = synth.gaussians(400, 31)
    p[:3, 0:3] = (cam.pos - 0.5 * cam.R[2].astype(np.float64)).astype(np.float32)
    rng = np.random.default_rng(4)
    m0 = rng.normal(0, 1e-3, p.shape).astype(np.float32)
    v0 = rng.uniform(1e-6, 1e-5, p.shape).astype(np.float32)
    target = torch.from_numpy(rng.uniform(0, 1, (3, 48, 64)).astype(np.float32)).cuda()
    ws = gpu.Workspace(400, 1 << 20, 64, 48)
    cfg = gpu.raster_cfg()
    adam = gpu.adam_params(gpu.PAPER_LR, step=3)
    out = []
    for with_grads in (True, False):
        P, M, V = (torch.from_numpy(a.copy()).cuda() for a in (p, m0, v0))
        view = dict(params=P, cam=cam, target=target, loss=torch.zeros((), device="cuda"), m=M, v=V)
        if with_grads:
            view["grads"] = torch.zeros_like(P)
        gpu.train_step([view], adam, cfg, ws, gpu.LOSS_HDR)
        ws.status()
        out.append([x.cpu().numpy() for x in (P, M, V)])
    for a, b in zip(out[0], out[1]):
        np.testing.assert_allclose(b, a, rtol=1e-4, atol=1e-6 * np.abs(a).max())
        np.testing.assert_array_equal(b[:3], a[:3])
    assert np.abs(out[1][0] - p).max() > 0


def test_batch_with_per_view_bins(gpu):
    """bin_size 0: every view of a batch bins at its own size (256^2 and
    640x480 at 32 px, 1280x720 at 64, 1920x1080 at 128); the images equal the
    single-view renders at a fixed 64-px bin bit for bit, and the gradients
    match to the order of the atomics."""
    import torch
    scene = torch.from_numpy(synth.gaussians(2000, 812)).cuda()
    res = [(256, 256), (640, 480), (1280, 720), (1920, 1080)]
    views = []
    for i, (w, h) in enumerate(res):
        views.append(dict(params=scene, cam=gpu.camera(synth.orbit_camera(w, h, 50.0 + 30.0 * i)),
                          image=torch.zeros((3, h, w), device="cuda"),
                          dL_dimage=torch.from_numpy(np.random.default_rng(60 + i).uniform(
                              -1, 1, (3, h, w)).astype(np.float32)).cuda()))
    grads = torch.zeros_like(scene)
    for v in views:
        v["grads"] = grads
    ws = gpu.Workspace(2000 * 4, 1 << 23, 1920, 1080, max_views=4)
    gpu.render_batch(views, gpu.BATCH_FWD | gpu.BATCH_BWD, gpu.raster_cfg(tile=(16, 16), pixels_per_thread=2), ws)
    ws.status()
    ref = torch.zeros_like(scene)
    alone = gpu.Workspace(2000, 1 << 23, 1920, 1080)
    fixed = gpu.raster_cfg(tile=(16, 16), bin_size=64, pixels_per_thread=2)
    for v in views:
        img = gpu.cache_render(v["params"], v["cam"], fixed, alone)
        gpu.cache_backward(v["params"], v["cam"], fixed, alone, v["dL_dimage"], ref)
        alone.status()
        assert torch.equal(img, v["image"])
        assert float(img.abs().max()) > 0
    g, r = grads.cpu().numpy(), ref.cpu().numpy()
    np.testing.assert_allclose(g, r, rtol=2e-3, atol=1e-5 * np.abs(r).max())
