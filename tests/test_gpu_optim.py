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
    np.testing.assert_allclose(grad.cpu().numpy(), rgrad, rtol=2e-6, atol=1e-12)


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
    orc.adamw(rp, rg, rm, rv, lr.astype(np.float64), 0.6, 0.9, 0.999, 1e-15, 0.01, 5)
    np.testing.assert_allclose(P.cpu().numpy().reshape(-1), rp, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(M.cpu().numpy().reshape(-1), rm, rtol=1e-5, atol=1e-10)
    np.testing.assert_allclose(V.cpu().numpy().reshape(-1), rv, rtol=1e-5, atol=1e-12)
    assert float(G.abs().max()) == 0.0
    frozen = np.tile(lr == 0, n)
    np.testing.assert_array_equal(P.cpu().numpy().reshape(-1)[frozen], p.reshape(-1)[frozen])
