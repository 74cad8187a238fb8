"""Comparisons of the CUDA path with the oracle that leave no pixel out.

A compositing decision (alpha >= alpha_min, the T_min stop, the alpha_max
clamp) that the FP64 oracle finds within 2e-4 (relative) of its threshold
may be taken the other way by FP32 arithmetic.  Instead of skipping such
pixels, the oracle enumerates every way they can go:

- forward: each pixel's value must lie within 1e-4 (every channel) of one
  of the pixel's possible results ("leaves");
- gradient: the 2D gradient record of a Gaussian lies, in exact arithmetic,
  in [lo, hi], the sums over pixels of the smallest and largest contribution
  among the pixel's leaves.  Its packed parameter gradient J a then lies in
  J mid +- M(rad) (mid, rad the centre and half-width, M(x) >= |J x| the
  projection backward evaluated on absolute values), which the GPU value
  must meet within 1e-3 |J mid| plus the rounding an FP32 evaluation may
  carry, (80 + 8 sqrt(n)) u M(m): m the summed largest absolute per-pixel
  contributions, n their number, u = 2^-24 (80 u for each term's own FP32
  arithmetic and the projection backward, whose intermediate values M also
  bounds, 8 sqrt(n) u for eight standard deviations of an n-term sum taken in
  an arbitrary order).
"""
import numpy as np

U = 2.0 ** -24


def fp32_sum_bar(orc, params, cam, abs2d, nterm, cfg=None):
    """(80 + 8 sqrt(n)) u M(m) per Gaussian and packed slot."""
    return (80.0 + 8.0 * np.sqrt(nterm))[:, None] * U * orc.grad_abs_map(params, cam, abs2d, cfg)


def assert_within_leaves(got, leaves, nleaves, tol=1e-4, what=""):
    """got (3, h, w): every pixel within tol of one of its leaves."""
    assert nleaves.min() >= 1, f"{what}: a pixel has more marginal decisions than the oracle enumerates"
    d = np.abs(leaves - np.asarray(got, np.float64).transpose(1, 2, 0)[:, :, None, :]).max(-1)
    d = np.where(np.arange(leaves.shape[2])[None, None, :] < nleaves[:, :, None], d, np.inf).min(-1)
    worst = np.unravel_index(np.argmax(d), d.shape)
    assert d.max() <= tol, (what, float(d.max()), worst, int(nleaves[worst]))
    return int((nleaves > 1).sum())


def render_check(orc, got, params, cam, window, cfg=None, tol=1e-4, what=""):
    """got = the GPU's image over window (x0, y0, w, h), against the leaves."""
    leaves, n = orc.render_leaves(params, cam, cfg, window=window)
    return assert_within_leaves(got, leaves, n, tol, what)


def grad_bounds(orc, params, cam, dl, cfg=None, window=None):
    """Centre and half-width of the packed gradient and the FP32 bar, for
    upstream gradient dl over window: (g_mid, g_rad, bar, nleaves)."""
    lo, hi, ab, nterm, nl = orc.render_backward_bounds(params, cam, dl, cfg, window=window)
    assert nl.min() >= 0 and not (nl < 0).any(), "a pixel has more marginal decisions than the oracle enumerates"
    g_mid = orc.project_backward(params, cam, 0.5 * (lo + hi), cfg)
    g_rad = orc.grad_abs_map(params, cam, 0.5 * (hi - lo), cfg)
    return g_mid, g_rad, fp32_sum_bar(orc, params, cam, ab, nterm, cfg), nl


def assert_grad_within(got, g_mid, g_rad, bar, rel=1e-3, what=""):
    """got (N, 16) packed gradient against the bounds of grad_bounds."""
    got = np.asarray(got, np.float64)
    bad = np.abs(got - g_mid) > g_rad + rel * np.abs(g_mid) + bar
    assert not bad.any(), (what, np.argwhere(bad)[:5].tolist(), got[bad][:5], g_mid[bad][:5], g_rad[bad][:5],
                           bar[bad][:5])
