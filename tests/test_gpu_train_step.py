"""The benchmarked training step (gsc_train_step: render, HDR loss and
backward of every cache level in one launch, then the per-Gaussian gradient
and the AdamW step in one more; Sec. 3.5-3.6) against the oracle's separate
definitions -- render, HDR loss, backward, AdamW -- at the benchmark's size:
1920x1080, 1M Gaussians in three levels (571,429 / 285,714 / 142,857), in
the launch configurations the frame loop runs (16x16 tiles at 4 pixels per
thread with a staging of 96 entries and 128-px bins, and the lower
pixels-per-thread candidates it switches to as the cache trains).

The gradient is confined to a 64x64 crop so that the oracle can follow it:
each level's target is its own render outside the crop (the HDR gradient is
then exactly zero there) and the render plus seeded noise inside it.
Checked, per level and launch configuration:
- the image the step writes: bit-identical to gsc_cache_render's, and on the
  crop and on sampled windows (the ragged bottom-right corner among them)
  every pixel within 1e-4 of a result the oracle allows (its own, and each way
  a decision within 2e-4 of a threshold can go);
- the loss against the oracle's HDR loss of the GPU's own image (2e-6);
- post-step p, m, v of every Gaussian the crop touches against the oracle's
  AdamW applied to the oracle's gradient: AdamW is monotone in the gradient
  for the moments used here (m = 0, v > 0 before the step), so the GPU value
  must lie between the oracle's outputs at the two ends of the gradient's
  bounds, widened by AdamW's own FP32 bound.  The gradient's bounds are the
  oracle's over every way a marginal decision of a crop pixel can go, plus
  1e-3 of their centre and the rounding an FP32 sum of the gradient's terms
  may carry (tests/parity.py);
- Gaussians the crop does not touch: the oracle's zero-gradient step.
"""
import numpy as np
import pytest

from parity import assert_grad_within, grad_bounds, render_check

from paper_2507_19718_gb300 import synth

pytestmark = pytest.mark.gpu

W, H = 1920, 1080
CROP = (928, 508, 64, 64)
WINDOWS = [(940, 300, 16, 16), (600, 700, 16, 16), (1904, 1064, 16, 16)]
B1, B2, EPS, WD, STEP = 0.9, 0.999, 1e-15, 0.01, 4
LAUNCHES = [dict(tile=(16, 16), list_capacity=96, bin_size=128, pixels_per_thread=4),
            dict(tile=(16, 16), list_capacity=128, bin_size=128, pixels_per_thread=2),
            dict(tile=(16, 16), list_capacity=256, bin_size=128, pixels_per_thread=1)]


def _f(x):
    return float(np.float32(x))


@pytest.fixture(scope="module")
def case(gpu, orc):
    """Levels, targets and the oracle's expected loss, gradient and AdamW
    inputs, shared by the launch configurations."""
    import torch
    sizes = synth.level_sizes(1_000_000, 3)
    assert sizes == [571_429, 285_714, 142_857]
    cam = synth.orbit_camera(W, H, 4.5)
    rng = np.random.default_rng(20250726)
    levels = [synth.gaussians(n, synth.BASE_SEED + 1000 + k) for k, n in enumerate(sizes)]
    ws = gpu.Workspace(sum(sizes), 48_000_000, W, H, max_views=3)
    x0, y0, cw, ch = CROP
    out = []
    for k, p in enumerate(levels):
        R = gpu.cache_render(torch.from_numpy(p).cuda(), cam, gpu.raster_cfg(), ws)
        ws.status()
        R = R.cpu().numpy()
        _, _, ncon, _ = orc.render(p, cam, window=CROP)
        assert ncon.mean() > 20, ncon.mean()
        tgt = R.copy()
        noise = R[:, y0:y0 + ch, x0:x0 + cw] * rng.uniform(-0.25, 0.25, (3, ch, cw)) + \
            rng.uniform(0.0, 0.02, (3, ch, cw))
        tgt[:, y0:y0 + ch, x0:x0 + cw] = (R[:, y0:y0 + ch, x0:x0 + cw] + noise).astype(np.float32)
        val, dl = orc.loss_hdr(R, tgt)
        outside = np.ones((3, H, W), bool)
        outside[:, y0:y0 + ch, x0:x0 + cw] = False
        assert np.all(dl[outside] == 0.0)
        g_mid, g_rad, bar, nl = grad_bounds(orc, p, cam, dl[:, y0:y0 + ch, x0:x0 + cw], window=CROP)
        assert (nl > 1).sum() > 0  # marginal pixels are in the comparison
        m0 = np.zeros_like(p)
        v0 = rng.uniform(1e-8, 1e-5, p.shape).astype(np.float32)
        out.append(dict(p=p, R=R, tgt=tgt, loss=val, g=g_mid, tol=g_rad + 1e-3 * np.abs(g_mid) + bar, m0=m0, v0=v0))
    return cam, out, ws


def _adam_ref(orc, p, g, m0, v0, lr):
    """Oracle AdamW with the FP32 hyper-parameters the kernel receives."""
    rp, rg, rm, rv = (np.ascontiguousarray(x, np.float64).reshape(-1) for x in (p, g, m0, v0))
    orc.adamw(rp, rg.copy(), rm, rv, np.asarray(lr, np.float64), 1.0, _f(B1), _f(B2), _f(EPS), _f(WD), STEP)
    return rp.reshape(p.shape), rm.reshape(p.shape), rv.reshape(p.shape)


@pytest.mark.parametrize("launch", LAUNCHES, ids=lambda d: f"ppt{d['pixels_per_thread']}_cap{d['list_capacity']}")
def test_train_step_matches_oracle_at_bench_scale(gpu, orc, case, launch):
    import torch
    cam, lv, ws = case
    cfg = gpu.raster_cfg(**launch)
    lr = gpu.PAPER_LR
    adam = gpu.adam_params(lr, beta1=B1, beta2=B2, eps=EPS, weight_decay=WD, lr_scale=1.0, step=STEP)
    views, state = [], []
    for k, L in enumerate(lv):
        P = torch.from_numpy(L["p"].copy()).cuda()
        M = torch.from_numpy(L["m0"].copy()).cuda()
        V = torch.from_numpy(L["v0"].copy()).cuda()
        img = torch.zeros((3, H, W), device="cuda")
        loss = torch.zeros((), device="cuda")
        views.append(dict(params=P, cam=cam, target=torch.from_numpy(L["tgt"]).cuda(), image=img, loss=loss,
                          m=M, v=V))
        state.append((P, M, V, img, loss))
    gpu.train_step(views, adam, cfg, ws, gpu.LOSS_HDR)
    ws.status()
    x0, y0, cw, ch = CROP
    for k, (L, (P, M, V, img, loss)) in enumerate(zip(lv, state)):
        image = img.cpu().numpy()
        # the step's image is the forward's, bit for bit
        np.testing.assert_array_equal(image, L["R"], err_msg=f"level {k}")
        # ... and the oracle's render, on the crop and on sampled windows
        render_check(orc, image[:, y0:y0 + ch, x0:x0 + cw], L["p"], cam, CROP, what=f"level {k} crop")
        for (wx, wy, ww, wh) in WINDOWS:
            ww, wh = min(ww, W - wx), min(wh, H - wy)
            render_check(orc, image[:, wy:wy + wh, wx:wx + ww], L["p"], cam, (wx, wy, ww, wh),
                         what=f"level {k} {(wx, wy)}")
        # the loss of the GPU's own image
        ref_loss, _ = orc.loss_hdr(image, L["tgt"])
        assert float(loss) == pytest.approx(ref_loss, rel=2e-6), k
        assert L["loss"] > 0

        # AdamW after the gradient: monotone in g here, so the GPU value lies
        # between the oracle's outputs at the ends of the gradient bar
        g = L["g"]
        touched = np.abs(g).sum(1) > 0
        assert touched.sum() > 200, touched.sum()
        tol = L["tol"]
        idx = np.nonzero(touched)[0]
        p_ref = L["p"][idx]
        lo = _adam_ref(orc, p_ref, g[idx] - tol[idx], L["m0"][idx], L["v0"][idx], lr)
        hi = _adam_ref(orc, p_ref, g[idx] + tol[idx], L["m0"][idx], L["v0"][idx], lr)
        zero = _adam_ref(orc, p_ref, np.zeros_like(g[idx]), L["m0"][idx], L["v0"][idx], lr)
        got_p = P.cpu().numpy().astype(np.float64)
        got_m = M.cpu().numpy().astype(np.float64)
        got_v = V.cpu().numpy().astype(np.float64)
        live = np.broadcast_to(lr > 0, g[idx].shape)
        p0 = p_ref.astype(np.float64)
        for name, got, a, b, extra, slack in [
                ("p", got_p[idx], lo[0], hi[0], None, 1e-6 * np.abs(p0) + 8e-6 * np.abs(lo[0] - p0) + 1e-9),
                ("m", got_m[idx], lo[1], hi[1], None, 4e-7 * np.abs(lo[1]) + 1e-30),
                ("v", got_v[idx], lo[2], hi[2], zero[2], 4e-7 * np.abs(lo[2]) + 1e-30)]:
            lo_b, hi_b = np.minimum(a, b), np.maximum(a, b)
            if extra is not None:  # v = b2 v0 + (1 - b2) g^2 is smallest at g = 0
                spans0 = (g[idx] - tol[idx] <= 0) & (g[idx] + tol[idx] >= 0)
                lo_b = np.where(spans0, np.minimum(lo_b, extra), lo_b)
            bad = live & ((got < lo_b - slack) | (got > hi_b + slack))
            assert not bad.any(), (k, name, np.argwhere(bad)[:5], got[bad][:5], lo_b[bad][:5], hi_b[bad][:5])
        # untouched Gaussians took the zero-gradient step
        rest = np.nonzero(~touched)[0][::97]
        zp, zm, zv = _adam_ref(orc, L["p"][rest], np.zeros((len(rest), 16)), L["m0"][rest], L["v0"][rest], lr)
        p0r = L["p"][rest].astype(np.float64)
        assert np.all(np.abs(got_p[rest] - zp) <= 1e-6 * np.abs(zp) + 8e-6 * np.abs(zp - p0r) + 1e-9)
        assert np.all(got_m[rest] == 0.0)
        assert np.all(np.abs(got_v[rest] - zv) <= 4e-7 * zv + 1e-30)


@pytest.mark.parametrize("tile,ppt", [((16, 16), 8), ((32, 8), 8), ((16, 16), 4), ((8, 8), 1)])
def test_feedback_order_and_split_change_no_result(gpu, orc, tile, ppt):
    """A gradient launch orders the next launch's tiles by the work it
    measured (same geometry) and splits the heaviest tiles into parts (up to
    4 with one-warp CTAs, 2 with larger ones, never more than a thread's
    pixels).  The training step's image and loss are the same bits on the
    first call (plain order) and on the later ones, the gradients agree up to
    the order of the FP32 atomics and match the oracle, and the split
    happened (more work items than tiles) exactly where it can: on this small
    frame the grid has 4 CTAs per tile, so every tile outlasts a CTA's mean
    load."""
    import torch
    w, h = 128, 96
    p = synth.gaussians(1024, synth.BASE_SEED + 2)
    cam = synth.orbit_camera(w, h, 30.0)
    cfg = gpu.raster_cfg(tile=tile, list_capacity=256, bin_size=64, pixels_per_thread=ppt)
    ws = gpu.Workspace(len(p), 1 << 21, w, h)
    P = torch.from_numpy(p).cuda()
    R = gpu.cache_render(P, cam, cfg, ws).cpu().numpy()
    rng = np.random.default_rng(7)
    tgt = (R * (1 + rng.uniform(-0.3, 0.3, R.shape)) + rng.uniform(0, 0.05, R.shape)).astype(np.float32)
    T = torch.from_numpy(tgt).cuda()
    tiles = (-(-w // tile[0])) * (-(-h // tile[1]))
    runs = []
    for call in range(3):
        G = torch.zeros_like(P)
        img = torch.zeros((3, h, w), device="cuda")
        loss = torch.zeros((), device="cuda")
        gpu.train_batch([dict(params=P, cam=cam, target=T, grads=G, loss=loss, image=img)], cfg, ws, gpu.LOSS_HDR)
        c = ws.counters()
        runs.append((img.cpu().numpy(), float(loss), G.cpu().numpy().astype(np.float64), c["items_last"]))
    can_split = ppt > 1
    assert runs[0][3] == tiles
    for img, lv, g, items in runs[1:]:
        np.testing.assert_array_equal(img, runs[0][0])
        assert lv == runs[0][1]
        np.testing.assert_allclose(g, runs[0][2], rtol=1e-5, atol=1e-6 * np.abs(runs[0][2]).max())
        assert (items > tiles) if can_split else (items == tiles), (items, tiles)
    # the split launch's gradient against the oracle's bounds, every pixel included
    _, dl = orc.loss_hdr(runs[2][0], tgt)
    g_mid, g_rad, bar, _ = grad_bounds(orc, p, cam, dl)
    assert np.abs(g_mid).max() > 0
    assert_grad_within(runs[2][2], g_mid, g_rad, bar)
