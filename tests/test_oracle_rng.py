"""Pins of the oracle's random-number generator and FP32 elementary functions.

Philox4x32-10 against the published known-answer vectors (Salmon et al.,
SC'11); the FP32-mirror ln / sincos(2 pi u) against libm within stated bounds.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(orc, ctr, key, expect):
    assert list(orc.philox4x32_10(ctr, key)) == expect


def test_ln_f32_accuracy(orc):
    rng = np.random.default_rng(3)
    # the tracer evaluates ln(1 - u) for u = k 2^-24, i.e. arguments in [2^-24, 1]
    x = np.concatenate([rng.uniform(2.0 ** -24, 1.0, 200000), (np.arange(1, 4097) * 2.0 ** -24),
                        1.0 - np.arange(0, 4096) * 2.0 ** -24]).astype(np.float32)
    y = orc.ln_f32(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    err = np.abs(y - ref)
    # a few ulp of the result, plus an absolute floor near ln(1) = 0
    assert np.all(err <= 3e-7 * np.abs(ref) + 2e-7), err.max()
    assert orc.ln_f32(np.array([1.0], np.float32))[0] == 0.0


def test_sincos2pi_f32_accuracy(orc):
    u = np.concatenate([np.random.default_rng(4).uniform(0, 1, 200000),
                        np.arange(0, 1 << 12) / float(1 << 12)]).astype(np.float32)
    s, c = orc.sincos2pi_f32(u)
    ref_s, ref_c = np.sin(2 * np.pi * u.astype(np.float64)), np.cos(2 * np.pi * u.astype(np.float64))
    assert np.max(np.abs(s - ref_s)) < 4e-7
    assert np.max(np.abs(c - ref_c)) < 4e-7
    # exact quadrant structure: u = 0 -> (0, 1), 0.25 -> (1, 0) ...
    s4, c4 = orc.sincos2pi_f32(np.array([0.0, 0.25, 0.5, 0.75], np.float32))
    np.testing.assert_allclose(s4, [0, 1, 0, -1], atol=3e-7)
    np.testing.assert_allclose(c4, [1, 0, -1, 0], atol=3e-7)


def test_sphere_directions_are_uniform(orc):
    """z = 1 - 2 u1 and phi = 2 pi u2 give unit vectors with zero mean and
    isotropic second moments (E[x^2] = E[y^2] = E[z^2] = 1/3)."""
    rng = np.random.default_rng(5)
    u1 = rng.uniform(0, 1, 400000).astype(np.float32)
    u2 = rng.uniform(0, 1, 400000).astype(np.float32)
    s, c = orc.sincos2pi_f32(u2)
    z = 1 - 2 * u1.astype(np.float64)
    r = np.sqrt(np.maximum(0, 1 - z * z))
    d = np.stack([r * c, r * s, z], 1)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1, atol=2e-6)
    np.testing.assert_allclose(d.mean(0), 0, atol=6e-3)
    np.testing.assert_allclose((d * d).mean(0), 1 / 3, atol=6e-3)
