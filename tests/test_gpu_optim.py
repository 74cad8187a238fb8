"""GPU losses (Sec. 3.6) and AdamW step against the FP64 oracle, through the
C ABI."""
import numpy as np
import pytest

from paper_2507_19718_gb300 import synth

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("kind,crop", [(0, None), (1, None), (0, (13, 7, 200, 91)), (1, (0, 0, 5, 3))])
def test_hdr_loss_matches_oracle(gpu, orc, kind, crop):
    rng = np.random.default_rng(kind)
    pred = rng.uniform(0.0, 2.0, (3, 120, 257)).astype(np.float32)
    tgt = (rng.uniform(0.0, 3.0, (3, 120, 257)) * (rng.uniform(size=(3, 120, 257)) < 0.5)).astype(np.float32)
    ws = gpu.Workspace(16, 16, 8, 8)
    val, grad = gpu.loss(kind, _t(pred), _t(tgt), ws, crop=crop)
    ref, rgrad = orc.loss_hdr(pred, tgt, crop=crop, full_grad=bool(kind))
    assert float(val) == pytest.approx(ref, rel=2e-6)
    # FP32 error of the largest term; the full-gradient variant cancels two terms
    np.testing.assert_allclose(grad.cpu().numpy(), rgrad, rtol=2e-6, atol=1e-6 * np.abs(rgrad).max())


def test_adamw_matches_oracle(gpu, orc):
    rng = np.random.default_rng(3)
    n = 100_003
    p = rng.normal(0, 1, (n, 16)).astype(np.float32)
    g = rng.normal(0, 1e-2, (n, 16)).astype(np.float32)
    m = rng.normal(0, 1e-3, (n, 16)).astype(np.float32)
    v = rng.uniform(0, 1e-4, (n, 16)).astype(np.float32)
    g[::7] = 0.0
    lr = np.array(gpu.PAPER_LR, np.float32)
    a = gpu.adam_params(lr, weight_decay=0.01, lr_scale=0.6, step=5)
    P, G, M, V = _t(p), _t(g), _t(m), _t(v)
    gpu.cache_step(P, G, M, V, a)
    rp, rg, rm, rv = (x.astype(np.float64).reshape(-1) for x in (p, g, m, v))
    # the kernel receives FP32 hyper-parameters; the oracle gets the same values
    f = lambda x: float(np.float32(x))  # noqa: E731
    orc.adamw(rp, rg, rm, rv, lr.astype(np.float64), f(0.6), f(0.9), f(0.999), f(1e-15), f(0.01), 5)
    # FP32 rounding of the update (a few ulp of |dp|) and of the final sum (of |p|)
    got = P.cpu().numpy().reshape(-1).astype(np.float64)
    dp = np.abs(rp - p.reshape(-1).astype(np.float64))
    bound = 1e-6 * np.abs(rp) + 8e-6 * dp + 1e-9
    assert np.all(np.abs(got - rp) <= bound), np.max(np.abs(got - rp) / bound)
    # moments: a few FP32 ulps of the two summed terms (they may cancel)
    g64, m64, v64 = (x.reshape(-1).astype(np.float64) for x in (g, m, v))
    live = np.tile(lr > 0, n)
    bm = 4e-7 * (np.abs(m64) + 0.1 * np.abs(g64)) + 1e-30
    bv = 4e-7 * (v64 + 0.001 * g64 * g64) + 1e-30
    gm, gv = M.cpu().numpy().reshape(-1), V.cpu().numpy().reshape(-1)
    assert np.all(np.abs(gm - rm)[live] <= bm[live])
    assert np.all(np.abs(gv - rv)[live] <= bv[live])
    np.testing.assert_array_equal(gm[~live], m.reshape(-1)[~live])
    assert float(G.abs().max()) == 0.0
    frozen = np.tile(lr == 0, n)
    np.testing.assert_array_equal(P.cpu().numpy().reshape(-1)[frozen], p.reshape(-1)[frozen])


@pytest.mark.parametrize("crop", [None, (13, 7, 200, 91), (0, 0, 9, 6)])
def test_l1ssim_loss_matches_oracle(gpu, orc, crop):
    rng = np.random.default_rng(21)
    tgt = synth.smooth_noisy_image(3, 120, 257, 5)
    pred = np.clip(tgt + rng.normal(0, 0.1, tgt.shape), 0, None).astype(np.float32)
    ws = gpu.Workspace(16, 16, 257, 120)
    val, grad = gpu.loss(gpu.LOSS_L1_SSIM, _t(pred), _t(tgt), ws, crop=crop)
    ref, rgrad, _ = orc.loss_l1ssim(pred, tgt, crop=crop)
    assert float(val) == pytest.approx(ref, rel=2e-5)
    g = grad.cpu().numpy()
    # the SSIM part sums 121-tap window moments in FP32 (variance = E[x^2] - mu^2)
    np.testing.assert_allclose(g, rgrad, rtol=1e-3, atol=1e-3 * np.abs(rgrad).max())
    if crop is not None:
        outside = np.ones_like(g, bool)
        outside[:, crop[1]:crop[1] + crop[3], crop[0]:crop[0] + crop[2]] = False
        assert np.all(g[outside] == 0)
