"""Truncated Gaussian noise -- oracle (test infrastructure).

Sec. 2.4: the noise components are standard normal, and values beyond three
standard deviations are *truncated* to +-3 (option (b), the one the paper
uses; Fig. "gaussianoptions", right panel).  Normals come from the Philox
words by the Box-Muller transform: u = (x + 1/2) 2^-32 in (0, 1),
z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1), and
likewise z2, z3 from (u2, u3).  Mapping: xi_x = z0, xi_y = z1, n_theta = z2.
"""
import math

import numpy as np

from . import philox

CLAMP = 3.0


def uniforms(words):
    return [(w.astype(np.float64) + 0.5) * (2.0 ** -32) for w in words]


def box_muller(u0, u1):
    r = np.sqrt(-2.0 * np.log(u0))
    return r * np.cos(2.0 * math.pi * u1), r * np.sin(2.0 * math.pi * u1)


def clamp(z):
    """Sec. 2.4 option (b): truncate to [-3, 3]."""
    return np.clip(z, -CLAMP, CLAMP)


def normals(ids, step, seed, replica=0, tag=philox.TAG_NOISE):
    """(xi_x, xi_y, n_theta, spare) for the given particle ids at `step`
    (tag: the fourth counter word, see oracle.philox.substep_tag)."""
    u = uniforms(philox.draw(ids, step, seed, replica, tag))
    z0, z1 = box_muller(u[0], u[1])
    z2, z3 = box_muller(u[2], u[3])
    return clamp(z0), clamp(z1), clamp(z2), clamp(z3)


def clamped_normal_variance(c: float = CLAMP) -> float:
    """E[clip(Z, -c, c)^2] for standard normal Z, in closed form:
    (1 - 2Q) - 2 c phi(c) + 2 c^2 Q with Q = P(Z > c)."""
    phi = math.exp(-0.5 * c * c) / math.sqrt(2.0 * math.pi)
    Q = 0.5 * math.erfc(c / math.sqrt(2.0))
    return (1.0 - 2.0 * Q) - 2.0 * c * phi + 2.0 * c * c * Q
