"""gsc_loss_noalloc: the HDR loss for callers that cannot allocate device
memory (or hand the library a workspace) when they call it -- for example a
plug-in inside an application that owns all device allocations, or a frame
loop that forbids allocation once it runs.  Its scratch is a fixed array
inside the library, so this test checks, through the C ABI, that it gives the
same loss and gradient as the workspace entry point on two calls in a row
(the second call must not see anything left over from the first), and that
it refuses an image larger than its scratch.

This file is collected last on purpose: it must pass both in a fresh process
and after every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _pair(seed, shape):
    rng = np.random.default_rng(seed)
    pred = rng.uniform(0.0, 2.0, shape).astype(np.float32)
    tgt = (rng.uniform(0.0, 3.0, shape) * (rng.uniform(size=shape) < 0.5)).astype(np.float32)
    return pred, tgt


@pytest.mark.parametrize("kind,crop", [(0, None), (1, (17, 9, 301, 77))])
def test_noalloc_loss_matches_workspace_loss_twice(gpu, kind, crop):
    import torch
    ws = gpu.Workspace(16, 16, 8, 8)
    for call, (seed, shape) in enumerate([(10, (3, 270, 480)), (11, (3, 123, 345))]):
        pred, tgt = _pair(seed + kind, shape)
        P, T = _t(pred), _t(tgt)
        ref_val, ref_grad = gpu.loss(kind, P, T, ws, crop=crop)
        val, grad = gpu.loss_noalloc(kind, P, T, crop=crop)
        torch.cuda.synchronize()
        r, g = float(ref_val), ref_grad.cpu().numpy()
        assert float(val) == pytest.approx(r, rel=2e-6), call
        np.testing.assert_allclose(grad.cpu().numpy(), g, rtol=2e-6, atol=1e-6 * np.abs(g).max())


def test_noalloc_loss_rejects_oversized_input(gpu):
    big = _t(np.zeros((3, 2048, 1366), np.float32))  # 8,392,704 elements > 8,388,608
    with pytest.raises(gpu.GscError) as e:
        gpu.loss_noalloc(0, big, big)
    assert e.value.status == gpu.GSC_ERR_CAPACITY
    assert "scratch" in str(e.value)
