"""Pins for the truncated Gaussian noise (Sec. 2.4)."""
import math

import numpy as np

from oracle import noise


def test_clamped_variance_closed_form_value():
    # E[clip(Z,-3,3)^2] by numerical quadrature of the normal density,
    # independent of the closed form used in the oracle
    z = np.linspace(-3.0, 3.0, 200001)
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)
    inner = np.trapezoid(z * z * pdf, z)
    tail = 2 * 9.0 * 0.5 * math.erfc(3.0 / math.sqrt(2.0))
    assert abs(noise.clamped_normal_variance() - (inner + tail)) < 1e-9
    assert abs(noise.clamped_normal_variance() - 0.99500728) < 1e-8


def test_normals_moments_and_clamp():
    n = 400000
    zx, zy, zt, z3 = noise.normals(np.arange(n), step=17, seed=3)
    for z in (zx, zy, zt, z3):
        assert z.max() <= 3.0 and z.min() >= -3.0
        assert abs(z.mean()) < 5 / math.sqrt(n)
        se = math.sqrt(2.0 / n)
        assert abs(z.var() - noise.clamped_normal_variance()) < 5 * se
    # the pairs (z0, z1) are uncorrelated
    assert abs(np.mean(zx * zy)) < 5 / math.sqrt(n)
    # clamping puts mass 2*Q(3) exactly at the bounds
    at_bound = np.mean(np.abs(zx) == 3.0)
    q = math.erfc(3 / math.sqrt(2))
    assert abs(at_bound - q) < 5 * math.sqrt(q / n)


def test_tail_probabilities_of_fig_normal():
    # Fig. "normal" (Sec. 2.4): P(|Z| <= 1, 2, 3) = 0.683, 0.954, 0.997
    n = 400000
    u = noise.uniforms(noise.philox.draw(np.arange(n), 1, seed=5))
    z0, _ = noise.box_muller(u[0], u[1])
    for k, p in ((1, 0.683), (2, 0.954), (3, 0.997)):
        assert abs(np.mean(np.abs(z0) <= k) - p) < 0.002
