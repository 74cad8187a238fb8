"""Pins of the oracle's losses (HDR loss of Sec. 3.6; 0.8 L1 + 0.2 D-SSIM),
AdamW step (Sec. 3.6 "Regularization") and learning-rate schedule (Eq. 4).

Closed forms for constant images and equal images; gradients against
central finite differences and (for the stop-gradient HDR variant, which is a
weighted L2 loss) against torch autograd in FP64; AdamW against
torch.optim.AdamW / Adam in FP64, which it must reduce to when every slot has
the same learning rate.
"""
import math

import numpy as np
import pytest

from paper_2507_19718_gb300 import synth


def _imgs(seed, shape=(3, 12, 14), lo=0.05, hi=1.0):
    r = np.random.default_rng(seed)
    return r.uniform(lo, hi, shape).astype(np.float32), r.uniform(0.0, 1.5, shape).astype(np.float32)


def test_hdr_closed_forms(orc):
    x = np.full((3, 5, 7), 0.7, np.float32)
    y = np.full((3, 5, 7), 0.2, np.float32)
    val, _ = orc.loss_hdr(y, x)
    xf, yf = float(np.float32(0.7)), float(np.float32(0.2))
    assert val == pytest.approx((xf - yf) ** 2 / (yf + 0.01) ** 2, rel=1e-12)
    v0, g0 = orc.loss_hdr(x, x)
    assert v0 == 0.0 and np.all(g0 == 0)


@pytest.mark.parametrize("full", [False, True])
def test_hdr_gradient(orc, full):
    torch = pytest.importorskip("torch")
    pred, tgt = _imgs(1)
    crop = (2, 3, 9, 6)
    val, g = orc.loss_hdr(pred, tgt, crop=crop, full_grad=full)
    yt = torch.tensor(pred, dtype=torch.float64, requires_grad=True)
    xt = torch.tensor(tgt, dtype=torch.float64)
    sl = (slice(None), slice(3, 9), slice(2, 11))
    den = yt[sl] + 0.01 if full else (yt[sl] + 0.01).detach()
    L = ((xt[sl] - yt[sl]) ** 2 / den ** 2).mean()
    L.backward()
    assert val == pytest.approx(L.item(), rel=1e-12)
    np.testing.assert_allclose(g, yt.grad.numpy(), rtol=1e-10, atol=1e-14)
    assert np.all(g[:, :3] == 0) and np.all(g[:, :, :2] == 0)


def test_hdr_full_gradient_matches_finite_differences(orc):
    pred, tgt = _imgs(2)
    _, g = orc.loss_hdr(pred, tgt, full_grad=True)
    rng = np.random.default_rng(0)
    for _ in range(20):
        idx = tuple(rng.integers(0, s) for s in pred.shape)
        h = 1e-4
        pp, pm = pred.copy(), pred.copy()
        pp[idx] = np.float32(pred[idx] + h)
        pm[idx] = np.float32(pred[idx] - h)
        heff = (float(pp[idx]) - float(pm[idx])) / 2
        fd = (orc.loss_hdr(pp, tgt)[0] - orc.loss_hdr(pm, tgt)[0]) / (2 * heff)
        assert fd == pytest.approx(g[idx], rel=1e-4, abs=1e-9)


def test_ssim_closed_forms(orc):
    x = synth.uniform_image(3, 20, 24, 5)
    v, g, smap = orc.loss_l1ssim(x, x)
    assert v == pytest.approx(0.0, abs=1e-12)
    np.testing.assert_allclose(smap, 1.0, atol=1e-9)
    # constant images p, q: away from the zero padding the local variances
    # vanish and SSIM = (2pq + C1) / (p^2 + q^2 + C1)
    p, q = np.float32(0.3), np.float32(0.8)
    a = np.full((3, 24, 24), p, np.float32)
    b = np.full((3, 24, 24), q, np.float32)
    v, _, smap = orc.loss_l1ssim(a, b)
    pf, qf = float(p), float(q)
    expect = (2 * pf * qf + 1e-4) / (pf * pf + qf * qf + 1e-4)
    np.testing.assert_allclose(smap[:, 5:-5, 5:-5], expect, rtol=1e-9)
    assert v == pytest.approx(0.8 * abs(pf - qf) + 0.2 * (1 - smap.mean()), rel=1e-12)


def test_l1ssim_gradient_matches_finite_differences(orc):
    pred, tgt = _imgs(3, (3, 16, 18))
    crop = (1, 2, 15, 12)
    _, g, _ = orc.loss_l1ssim(pred, tgt, crop=crop)
    rng = np.random.default_rng(1)
    n = 0
    while n < 24:
        idx = (int(rng.integers(0, 3)), int(rng.integers(2, 14)), int(rng.integers(1, 16)))
        if abs(float(pred[idx]) - float(tgt[idx])) < 1e-2:
            continue  # |.| kink of the L1 term
        h = 1e-3
        pp, pm = pred.copy(), pred.copy()
        pp[idx] = np.float32(pred[idx] + h)
        pm[idx] = np.float32(pred[idx] - h)
        heff = (float(pp[idx]) - float(pm[idx])) / 2
        fd = (orc.loss_l1ssim(pp, tgt, crop=crop)[0] - orc.loss_l1ssim(pm, tgt, crop=crop)[0]) / (2 * heff)
        assert fd == pytest.approx(g[idx], rel=1e-4, abs=1e-9), idx
        n += 1
    assert np.all(g[:, 0:2] == 0) and np.all(g[:, :, 0] == 0)


def test_l1ssim_crop_is_its_own_image(orc):
    pred, tgt = _imgs(4, (3, 20, 22))
    crop = (3, 4, 13, 11)
    v1, g1, _ = orc.loss_l1ssim(pred, tgt, crop=crop)
    v2, g2, _ = orc.loss_l1ssim(pred[:, 4:15, 3:16].copy(), tgt[:, 4:15, 3:16].copy())
    assert v1 == pytest.approx(v2, rel=1e-13)
    np.testing.assert_allclose(g1[:, 4:15, 3:16], g2, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("wd", [0.0, 0.01])
def test_adamw_reduces_to_torch(orc, wd):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    n = 64 * 16
    p = rng.normal(0, 1, n)
    m, v = np.zeros(n), np.zeros(n)
    lr = 3e-3
    tp = torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True)
    opt = (torch.optim.AdamW([tp], lr=lr, betas=(0.9, 0.999), eps=1e-15, weight_decay=wd) if wd
           else torch.optim.Adam([tp], lr=lr, betas=(0.9, 0.999), eps=1e-15))
    for step in range(1, 5):
        g = rng.normal(0, 1, n)
        tp.grad = torch.tensor(g.copy(), dtype=torch.float64)
        opt.step()
        gg = g.copy()
        orc.adamw(p, gg, m, v, np.full(16, lr), 1.0, 0.9, 0.999, 1e-15, wd, step)
        assert np.all(gg == 0)
    st = opt.state[tp]
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(m, st["exp_avg"].numpy(), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(v, st["exp_avg_sq"].numpy(), rtol=1e-12, atol=1e-15)


def test_adamw_first_step_closed_form_and_frozen_slots(orc):
    rng = np.random.default_rng(8)
    n = 8 * 16
    p0 = rng.normal(0, 1, n)
    g = rng.normal(0, 1, n)
    lr = np.array([1.16e-3, 1.16e-3, 1.16e-3, 1.5e-1, 0, 0, 0, 0, 1e-3, 1e-3, 1e-3, 1e-3, 1.25e-2, 1.25e-2,
                   1.25e-2, 0.0])
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    gg = g.copy()
    orc.adamw(p, gg, m, v, lr, 0.5, 0.9, 0.999, 1e-15, 0.01, 1)
    lre = np.tile(lr, 8) * 0.5
    # step 1: m_hat = g, v_hat = g^2, so the update is lr (sign(g) + wd p)
    expect = np.where(lre > 0, p0 - lre * (g / (np.abs(g) + 1e-15) + 0.01 * p0), p0)
    np.testing.assert_allclose(p, expect, rtol=1e-12, atol=1e-15)
    assert np.all(p[np.tile(lr, 8) == 0] == p0[np.tile(lr, 8) == 0])
    assert np.all(gg == 0)


def test_lr_schedule(orc):
    # Eq. 4: eta_t = eta_0 / (1 + log t); t = 1 on the first frame of a viewport
    assert orc.lr_scale(1) == 1.0
    assert orc.lr_scale(2) == pytest.approx(1 / (1 + math.log(2)), rel=1e-15)
    vals = [orc.lr_scale(t) for t in range(1, 200)]
    assert all(a > b for a, b in zip(vals, vals[1:]))
