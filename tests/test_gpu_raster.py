"""GPU parity of the Gaussian-splatting render and its gradient (Sec. 3.1,
Sec. 3.5) against the FP64 oracle, through the C ABI.

Every pixel is compared.  Forward: within 1e-4 absolute per channel of one
of the results the oracle allows, which is its own where no compositing
decision lies within 2e-4 of a threshold, and each way such a decision can go
where one does.  Tile size and staging capacity do not change a single bit.
Backward: dL/dimage random on every pixel, the packed gradient within the
oracle's bounds over those ways, 1e-3 of the centre and the rounding bar of an
FP32 sum of the gradient's terms (tests/parity.py).
"""
import numpy as np
import pytest
from parity import assert_grad_within, assert_within_leaves, grad_bounds, render_check

from paper_2507_19718_gb300 import synth

pytestmark = pytest.mark.gpu



def _torch():
    import torch
    return torch


def _ws(gsc, n, pairs, w, h):
    return gsc.Workspace(n, pairs, w, h)


def _render(gsc, p_np, cam, cfg, ws):
    torch = _torch()
    p = torch.from_numpy(p_np).cuda()
    img = gsc.cache_render(p, cam, cfg, ws)
    ws.status()
    return img.cpu().numpy().astype(np.float64)


def _scene0(n=1024, w=128, h=128, angle=30.0, seed=synth.BASE_SEED + 2):
    return synth.gaussians(n, seed), synth.orbit_camera(w, h, angle)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_render_matches_oracle_config0(gpu, orc, tile):
    p, cam = _scene0()
    ws = _ws(gpu, len(p), 1 << 21, cam.width, cam.height)
    img = _render(gpu, p, cam, gpu.raster_cfg(tile=tile), ws)
    ref, marg, ncon, _ = orc.render(p, cam)
    assert ncon.max() > 20 and ref.max() > 0.3 and marg.sum() > 0
    render_check(orc, img, p, cam, (0, 0, cam.width, cam.height), what=str(tile))


def test_tile_and_capacity_do_not_change_bits(gpu, orc):
    p, cam = _scene0(angle=75.0)
    ws = _ws(gpu, len(p), 1 << 22, cam.width, cam.height)
    base = _render(gpu, p, cam, gpu.raster_cfg(tile=(16, 16), list_capacity=256), ws)
    for tile, cap, b, ppt in [((8, 8), 64, 32, 1), ((32, 8), 2048, 64, 1), ((16, 8), 32, 128, 1),
                              ((8, 16), 512, 256, 1), ((8, 32), 128, 64, 1), ((32, 4), 96, 32, 1),
                              ((16, 16), 1024, 512, 1), ((16, 16), 256, 48, 1), ((16, 16), 128, 128, 2),
                              ((32, 8), 512, 64, 2), ((16, 8), 64, 32, 2), ((8, 32), 256, 128, 2),
                              ((16, 16), 64, 64, 4), ((32, 8), 256, 128, 4), ((8, 32), 32, 32, 4),
                              ((16, 16), 32, 128, 8), ((32, 8), 512, 64, 8), ((8, 32), 256, 256, 8)]:
        cfg = gpu.raster_cfg(tile=tile, list_capacity=cap, bin_size=b, pixels_per_thread=ppt)
        other = _render(gpu, p, cam, cfg, ws)
        np.testing.assert_array_equal(other, base, err_msg=str((tile, cap, b, ppt)))


def test_ragged_image_and_degenerate_gaussians(gpu, orc):
    # image size not a multiple of the tile; Gaussians behind the camera, off
    # screen, transparent, with a zero quaternion, and one covering the frame
    p, cam = _scene0(n=300, w=100, h=75, angle=200.0, seed=9)
    fwd = cam.R[2].astype(np.float64)
    p[0, 0:3] = (cam.pos - 0.5 * fwd).astype(np.float32)   # behind the camera
    p[1, 0:3] = (cam.pos + 0.1 * fwd).astype(np.float32)   # before the near plane
    p[2, 0:3] = (cam.pos + 2.0 * fwd + 5.0 * cam.R[0]).astype(np.float32)  # off screen
    p[3, 3] = -9.0                                          # opacity below alpha_min
    p[4, 8:12] = 0.0                                        # degenerate rotation
    p[5, 0:3] = (cam.pos + 1.2 * fwd).astype(np.float32)
    p[5, 4:7] = -0.3                                        # huge: covers the frame
    p[5, 3] = -2.0
    ws = _ws(gpu, len(p), 1 << 20, cam.width, cam.height)
    leaves, nl = orc.render_leaves(p, cam)
    for tile in [(16, 16), (8, 8), (32, 8)]:
        img = _render(gpu, p, cam, gpu.raster_cfg(tile=tile), ws)
        assert_within_leaves(img, leaves, nl, what=str(tile))
    ref, _, _, _ = orc.render(p, cam)
    assert ref[:, 0, 0].sum() > 0  # the big Gaussian reaches the corner


def test_empty_and_single(gpu, orc):
    torch = _torch()
    p, cam = _scene0(n=1, w=40, h=24, seed=4)
    p[0, 0:3] = [0.5, 0.5, 0.5]
    p[0, 4:7] = -2.0
    ws = _ws(gpu, 4, 1 << 12, cam.width, cam.height)
    img = _render(gpu, p, cam, gpu.raster_cfg(), ws)
    render_check(orc, img, p, cam, (0, 0, cam.width, cam.height))
    out = torch.full((3, cam.height, cam.width), 7.0, device="cuda")
    gpu.cache_render(torch.zeros((0, 16), device="cuda"), cam, gpu.raster_cfg(), ws, image=out)
    assert float(out.abs().max()) == 0.0


def test_pair_capacity_overflow_is_reported(gpu):
    torch = _torch()
    p, cam = _scene0()
    ws = _ws(gpu, len(p), 1000, cam.width, cam.height)
    img = gpu.cache_render(torch.from_numpy(p).cuda(), cam, gpu.raster_cfg(), ws)
    with pytest.raises(gpu.GscError) as e:
        ws.status()
    assert e.value.status == gpu.GSC_ERR_CAPACITY
    assert float(img.abs().max()) == 0.0  # nothing was composited, nothing overran
    need = _ws(gpu, len(p), 1 << 21, cam.width, cam.height)
    gpu.cache_render(torch.from_numpy(p).cuda(), cam, gpu.raster_cfg(), need)
    n = need.status()
    assert 1000 < n < (1 << 21)


@pytest.mark.parametrize("tile,ppt", [((16, 16), 1), ((8, 8), 1), ((16, 16), 2), ((32, 8), 2), ((16, 16), 4),
                                      ((8, 32), 4), ((16, 16), 8), ((32, 8), 8)])
def test_backward_matches_oracle_config0(gpu, orc, tile, ppt):
    torch = _torch()
    p, cam = _scene0(w=96, h=80)
    dL = np.random.default_rng(5).uniform(-1, 1, (3, cam.height, cam.width)).astype(np.float32)
    g_mid, g_rad, bar, nl = grad_bounds(orc, p, cam, dL.astype(np.float64))
    assert (nl > 1).sum() > 0  # marginal pixels are in the comparison
    ws = _ws(gpu, len(p), 1 << 21, cam.width, cam.height)
    g = gpu.cache_backward(torch.from_numpy(p).cuda(), cam, gpu.raster_cfg(tile=tile, pixels_per_thread=ppt), ws,
                           torch.from_numpy(dL).cuda())
    ws.status()
    g = g.cpu().numpy().astype(np.float64)
    assert np.all(g[:, [7, 15]] == 0)
    assert np.abs(g_mid).max() > 0
    assert_grad_within(g, g_mid, g_rad, bar, what=str((tile, ppt)))


def test_backward_accumulates_and_autograd_matches(gpu, orc):
    torch = _torch()
    p, cam = _scene0(n=400, w=64, h=48, seed=12)
    ws = _ws(gpu, len(p), 1 << 20, cam.width, cam.height)
    cfg = gpu.raster_cfg()
    params = torch.from_numpy(p).cuda().requires_grad_(True)
    w = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, (3, 48, 64)).astype(np.float32)).cuda()
    img = gpu.render(params, cam, cfg, ws)
    (img * w).sum().backward()
    direct = gpu.cache_backward(params.detach(), cam, cfg, ws, w)
    np.testing.assert_allclose(params.grad.cpu().numpy(), direct.cpu().numpy(), rtol=1e-5, atol=1e-7)
    twice = gpu.cache_backward(params.detach(), cam, cfg, ws, w, grads=direct.clone())
    np.testing.assert_allclose(twice.cpu().numpy(), 2 * direct.cpu().numpy(), rtol=1e-5, atol=1e-7)


def test_full_size_1080p_1M_sampled(gpu, orc):
    """At the benchmark's size (1920x1080, 1M Gaussians, 16x16 tiles):
    sampled windows of the image against the oracle, and the gradient of a
    loss living on a 32x32 crop against the oracle's crop gradient."""
    torch = _torch()
    n = 1_000_000
    p = synth.gaussians(n, synth.BASE_SEED + 3)
    cam = synth.orbit_camera(1920, 1080, 20.0)
    ws = _ws(gpu, n, 400_000_000, 1920, 1080)
    cfg = gpu.raster_cfg()
    params = torch.from_numpy(p).cuda()
    img = gpu.cache_render(params, cam, cfg, ws)
    need = ws.status()
    assert need > 5_000_000  # a full-size binning (7.7M pairs with the ellipses' own bounding boxes)
    img = img.cpu().numpy()
    marginal = 0
    for (x0, y0) in [(940, 520), (700, 300), (1300, 800), (0, 0)]:
        marginal += render_check(orc, img[:, y0:y0 + 16, x0:x0 + 16], p, cam, (x0, y0, 16, 16), what=str((x0, y0)))
    assert marginal > 0
    crop = (944, 524, 32, 32)
    dl = np.random.default_rng(2).uniform(-1, 1, (3, 32, 32)).astype(np.float32)
    full = np.zeros((3, 1080, 1920), np.float32)
    full[:, 524:556, 944:976] = dl
    g_mid, g_rad, bar, _ = grad_bounds(orc, p, cam, dl.astype(np.float64), window=crop)
    g = gpu.cache_backward(params, cam, cfg, ws, torch.from_numpy(full).cuda())
    ws.status()
    g = g.cpu().numpy().astype(np.float64)
    touched = np.abs(g_mid).sum(1) > 0
    assert touched.sum() > 100
    assert not np.abs(g[~touched]).any()
    assert_grad_within(g, g_mid, g_rad, bar)


def test_work_counters_count_the_composited_pairs(gpu, orc):
    """The roofline's numerator comes from device counters: the forward's
    composited pairs equal the oracle's per-pixel term counts (up to the
    marginal pixels), and the backward's re-walk and back-to-front phases
    count the same pairs."""
    torch = _torch()
    p, cam = _scene0(w=96, h=80, angle=50.0)
    ref, marg, ncon, _ = orc.render(p, cam)
    ws = _ws(gpu, len(p), 1 << 21, cam.width, cam.height)
    ws.counters()
    for tile, ppt in [((16, 16), 2), ((8, 32), 8)]:
        cfg = gpu.raster_cfg(tile=tile, pixels_per_thread=ppt)
        params = torch.from_numpy(p).cuda()
        gpu.cache_render(params, cam, cfg, ws)
        dl = torch.full((3, cam.height, cam.width), 1e-3, device="cuda")
        gpu.cache_backward(params, cam, cfg, ws, dl)
        c = ws.counters()
        assert abs(c["composited_fwd"] - int(ncon.sum())) <= 2 * int(marg.sum()) + 2, (c, int(ncon.sum()))
        assert c["composited_rewalk"] == c["composited_fwd"] == c["hits_back"]
        assert c["eval_rewalk"] == c["eval_fwd"] >= c["eval_back"] >= c["composited_fwd"] > 0
        assert c["binnings"] == 2 and c["pairs_sum"] > 0


def test_bin_culling_drops_only_unreachable_pairs(gpu, orc):
    """Long thin Gaussians (one axis e^-1.2, two e^-4.5, random rotations)
    have tile rectangles much larger than their ellipses: the binning lists
    a pair only in the bins of the rectangle that the falloff bound can
    reach.  Culling does drop pairs at every bin size, and the images at bin
    32, 64 and 128 (different culled sets) are the same bits and match the
    oracle on every pixel."""
    p = synth.gaussians(600, synth.BASE_SEED + 41)
    rng = np.random.default_rng(43)
    p[:, 4:7] = np.float32(-4.5)
    p[np.arange(len(p)), 4 + rng.integers(0, 3, len(p))] = np.float32(-1.2)
    cam = synth.orbit_camera(320, 240, 20.0)
    ws = _ws(gpu, len(p), 1 << 22, cam.width, cam.height)
    ws.counters()
    imgs = []
    for b in (32, 64, 128):
        imgs.append(_render(gpu, p, cam, gpu.raster_cfg(tile=(16, 16), bin_size=b), ws))
        c = ws.counters()
        assert 0 < c["pairs_culled"] < c["pairs_last"], (b, c)
    for img in imgs[1:]:
        np.testing.assert_array_equal(img, imgs[0])
    render_check(orc, imgs[0], p, cam, (0, 0, cam.width, cam.height))


def test_nine_bit_pair_sort_gives_the_same_bits(gpu, orc):
    """300 coarse bins (bin 32 on 640x480) are sorted in one 9-bit radix pass,
    20 bins (bin 128) in one 8-bit pass: the images are bit-identical, and
    the 9-bit case matches the oracle on sampled windows."""
    p, cam = _scene0(n=3000, w=640, h=480, angle=15.0, seed=31)
    ws = _ws(gpu, len(p), 1 << 22, cam.width, cam.height)
    nine = _render(gpu, p, cam, gpu.raster_cfg(tile=(16, 16), bin_size=32), ws)
    eight = _render(gpu, p, cam, gpu.raster_cfg(tile=(16, 16), bin_size=128), ws)
    np.testing.assert_array_equal(nine, eight)
    for (x0, y0) in [(300, 220), (0, 0), (624, 464)]:
        render_check(orc, nine[:, y0:y0 + 16, x0:x0 + 16], p, cam, (x0, y0, 16, 16), what=str((x0, y0)))


def _deep_stack(n=4000, w=32, h=32, seed=71):
    """n faint Gaussians spread over a small image in front of the camera:
    every 16x16 tile keeps about 2,900 of them, its pixels composite 400 to
    1,000 each, so the backward's hit ring wraps (earlier chunks are rebuilt
    from their recorded list positions)."""
    rng = np.random.default_rng(seed)
    p = synth.gaussians(n, seed)
    cam = synth.orbit_camera(w, h, 40.0)
    R = cam.R.astype(np.float64)
    depth = 2.2 + rng.uniform(-0.3, 0.3, n)
    xy = rng.uniform(-0.9, 0.9, (n, 2))
    p[:, 0:3] = (cam.pos + depth[:, None] * R[2] + xy[:, :1] * R[0] + xy[:, 1:] * R[1]).astype(np.float32)
    p[:, 4:7] = np.float32(-1.08) + rng.normal(0, 0.05, (n, 3)).astype(np.float32)
    p[:, 3] = np.float32(np.log(0.02 / 0.98))
    return p, cam


def test_deep_lists_wrap_the_hit_ring(gpu, orc):
    torch = _torch()
    p, cam = _deep_stack()
    _, _, ncon, _ = orc.render(p, cam)
    assert ncon.max() > 900 and ncon.min() > 300  # per-pixel composited terms
    ws = _ws(gpu, len(p), 1 << 20, cam.width, cam.height)
    params = torch.from_numpy(p).cuda()
    dL = np.random.default_rng(8).uniform(-1, 1, (3, cam.height, cam.width)).astype(np.float32)
    leaves, nl = orc.render_leaves(p, cam)
    assert (nl > 1).mean() > 0.05  # a pixel tests thousands of alphas: many have one within the margin
    g_mid, g_rad, bar, _ = grad_bounds(orc, p, cam, dL.astype(np.float64))
    for tile, ppt in [((16, 16), 4), ((8, 8), 1), ((32, 8), 2)]:
        cfg = gpu.raster_cfg(tile=tile, pixels_per_thread=ppt)
        img = gpu.cache_render(params, cam, cfg, ws)
        assert_within_leaves(img.cpu().numpy(), leaves, nl, what=str(tile))
        g = gpu.cache_backward(params, cam, cfg, ws, torch.from_numpy(dL).cuda())
        ws.status()
        assert_grad_within(g.cpu().numpy().astype(np.float64), g_mid, g_rad, bar, what=str((tile, ppt)))
