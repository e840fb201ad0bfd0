"""Euler-Maruyama update with active self-propulsion and walls -- oracle.

Eq. (integration), Sec. 2.2:  r(t+dt) = r(t) + F dt + xi * amp, with the
forces already in velocity units (mobility absorbed).  The active Brownian
model of Sec. 7 adds V0 (cos theta, sin theta) dt to the displacement and
diffuses the director as theta(t+dt) = theta + sqrt(2 D_r dt) n.

Noise amplitude: Eq. (integration) prints sqrt(D dt) while the rotational
update of Sec. 7 uses sqrt(2 D dt); the translational amplitude is read
here as sqrt(2 D dt) per component (mean-square displacement 4 D t in
2D); the literal sqrt(D dt) is kept behind `literal_amp=True`.

Walls (the paper's box is periodic, Sec. 2.1, kept as an option; the
benchmark configurations use reflecting walls): centres live in
[a, L - a]; a coordinate below a is mirrored to
2a - x, one above L - a to 2(L - a) - x.
"""
import math

import numpy as np

from . import noise, philox


def noise_amplitude(D, dt, literal_amp=False):
    return math.sqrt(D * dt) if literal_amp else math.sqrt(2.0 * D * dt)


def reflect(xy, a, L):
    """Mirror centres into [a, L - a]; a is the radius, or one radius per disk
    (polydisperse disks: each centre stays a_i from the walls)."""
    xy = np.array(xy, dtype=np.float64, copy=True)
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    lo, hi = a, L - a
    xy = np.where(xy < lo, 2.0 * lo - xy, xy)
    xy = np.where(xy > hi, 2.0 * hi - xy, xy)
    return xy


def em_move(xy, theta, F, ids, step, seed, D, Dr, v0, dt, replica=0, literal_amp=False,
            tag=philox.TAG_NOISE):
    """The Euler-Maruyama + ABP move before the walls.  Returns (xy', theta').
    dt is the length of this move (a piece of a redone step uses its own, with
    the noise of counter word `tag`)."""
    xi_x, xi_y, n_th, _ = noise.normals(ids, step, seed, replica, tag)
    amp = noise_amplitude(D, dt, literal_amp)
    th = np.asarray(theta, dtype=np.float64)
    dx = dt * (F[:, 0] + v0 * np.cos(th)) + amp * xi_x
    dy = dt * (F[:, 1] + v0 * np.sin(th)) + amp * xi_y
    new = np.stack([xy[:, 0] + dx, xy[:, 1] + dy], axis=1)
    th_new = th + math.sqrt(2.0 * Dr * dt) * n_th
    return new, th_new


def em_step(xy, theta, F, ids, step, seed, D, Dr, v0, dt, a, L, replica=0, literal_amp=False,
            tag=philox.TAG_NOISE):
    """One Euler-Maruyama + ABP step with reflection.  Returns (xy', theta')."""
    new, th_new = em_move(xy, theta, F, ids, step, seed, D, Dr, v0, dt, replica, literal_amp, tag)
    return reflect(new, a, L), th_new
