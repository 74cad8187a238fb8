"""Differentiation check at scale: the backward kernel for 1M Gaussians at
1920x1080 (FP32), through the C ABI, against the FP64 oracle on a 256x256
crop and against central finite differences (h = 1e-3) of 64 seeded
parameters spread over all 14 parameter kinds.

Workload: target = the oracle's render of the unperturbed cloud on the crop
plus N(0, 0.05^2) per element; evaluated parameters = the same cloud with
means jittered by N(0, 0.005^2); L1 + D-SSIM (0.8 / 0.2) over the crop at
(832, 412).  Every pixel of the crop is compared: the forward against the
results the oracle allows (its own, and each way a decision within 2e-4 of a
threshold can go), the gradient of the upstream gradient v = dL/dimage (the
oracle's, both backwards get the same v) against the oracle's bounds over
those ways (tests/parity.py).  The finite differences are those of
sum(v * render) with the oracle's threshold decisions frozen, which is the
function whose gradient the backward computes, taken with v zeroed on the
marginal pixels; a Richardson step (h and h/2) removes their O(h^2)
truncation.
"""
import numpy as np
import pytest
from parity import assert_grad_within, grad_bounds, render_check

from paper_2507_19718_gb300 import synth

pytestmark = pytest.mark.gpu

N = 1_000_000
W, H = 1920, 1080
CROP = (832, 412, 256, 256)
SLOTS = [0, 1, 2, 3, 4, 5, 6, 8, 9, 10, 11, 12, 13, 14]


def _within(got, ref, scale, rel=1e-3, floor=1e-3):
    """the finite-difference comparison: rel, down to floor x the slot's largest gradient"""
    return np.abs(got - ref) <= rel * np.maximum(np.abs(ref), floor * scale)


@pytest.fixture(scope="module")
def workload(orc):
    rng = np.random.default_rng(synth.BASE_SEED + 22)
    p_true = synth.gaussians(N, synth.BASE_SEED + 2)
    cam = synth.orbit_camera(W, H, 0.0)
    clean, _, _, _ = orc.render(p_true, cam, window=CROP)
    x0, y0, w, h = CROP
    target = np.zeros((3, H, W), np.float32)
    target[:, y0:y0 + h, x0:x0 + w] = clean + rng.normal(0.0, 0.05, clean.shape)
    p = p_true.copy()
    p[:, 0:3] += rng.normal(0.0, 0.005, (N, 3)).astype(np.float32)
    ref_img, marg, _, _ = orc.render(p, cam, window=CROP, grad_margins=True)
    loss, dl, _ = orc.loss_l1ssim(ref_img.astype(np.float32), target[:, y0:y0 + h, x0:x0 + w])
    v = dl.astype(np.float32)
    v_fd = v.copy()
    v_fd[:, marg] = 0.0
    return dict(p=p, cam=cam, target=target, ref_img=ref_img, marg=marg, loss=loss, v=v, v_fd=v_fd)


def test_config2_backward_vs_oracle_and_finite_differences(gpu, orc, workload):
    import torch
    p, cam, v = workload["p"], workload["cam"], workload["v"]
    x0, y0, w, h = CROP
    ws = gpu.Workspace(N, 400_000_000, W, H)
    cfg = gpu.raster_cfg(tile=(16, 16), list_capacity=256, bin_size=64, pixels_per_thread=2)
    params = torch.from_numpy(p).cuda()
    img = gpu.cache_render(params, cam, cfg, ws)
    ws.status()

    # forward on the crop: every pixel within 1e-4 of a result the oracle allows
    assert workload["marg"].mean() < 0.2, workload["marg"].mean()
    got = img[:, y0:y0 + h, x0:x0 + w].cpu().numpy()
    assert render_check(orc, got, p, cam, CROP) > 0

    # the loss kernel on the GPU's own image agrees with the oracle's loss
    val, _ = gpu.loss(gpu.LOSS_L1_SSIM, img, torch.from_numpy(workload["target"]).cuda(), ws, crop=CROP)
    assert abs(float(val) - workload["loss"]) <= 1e-3 * abs(workload["loss"])

    # backward with the same upstream gradient, on every pixel of the crop
    def backward(vv):
        full = np.zeros((3, H, W), np.float32)
        full[:, y0:y0 + h, x0:x0 + w] = vv
        gg = gpu.cache_backward(params, cam, cfg, ws, torch.from_numpy(full).cuda())
        ws.status()
        return gg.cpu().numpy().astype(np.float64)
    g = backward(v)
    g_mid, g_rad, bar, _ = grad_bounds(orc, p, cam, v.astype(np.float64), window=CROP)
    touched = np.abs(g_mid).sum(1) > 0
    assert touched.sum() > 2000
    assert not np.abs(g[~touched]).any()
    assert_grad_within(g, g_mid, g_rad, bar)

    # finite differences of the frozen-decision render, with v zeroed on the
    # marginal pixels (where frozen FP64 decisions and FP32 may part)
    v = workload["v_fd"]
    g = backward(v)
    ref, _ = orc.render_backward(p, cam, v.astype(np.float64), window=CROP)

    # 64 parameters: about 4-5 per kind, each on a Gaussian where that kind's
    # gradient is among the largest (and colours away from their clamp at 0)
    rng = np.random.default_rng(synth.BASE_SEED + 23)
    gauss, slots = [], []
    idx = np.nonzero(touched)[0]
    for k in range(64):
        s = SLOTS[k % len(SLOTS)]
        cand = idx[np.argsort(-np.abs(ref[idx, s]))[:500]]
        if s >= 12:
            cand = cand[p[cand, s] > 4e-3]
        gauss.append(int(rng.choice(cand)))
        slots.append(s)
    gauss, slots = np.array(gauss), np.array(slots)
    fl = orc.FrozenLists(p, cam, window=CROP)
    v64 = v.astype(np.float64)
    d1 = fl.fd(p, v64, gauss, slots, h=1e-3)
    d2 = fl.fd(p, v64, gauss, slots, h=5e-4)
    fd = (4.0 * d2 - d1) / 3.0
    an_o, an_g = ref[gauss, slots], g[gauss, slots]
    scale = np.array([np.abs(ref[touched][:, s]).max() for s in slots])
    assert _within(an_o, fd, scale, 1e-4).all(), np.abs(an_o - fd).max()
    assert _within(an_g, fd, scale).all(), np.abs(an_g - fd).max()
    assert _within(d1, fd, scale, 2e-2).all()  # the plain h = 1e-3 difference, within its truncation
