"""Independent 8-D dual-quaternion algebra for the tests (Kavan et al. blending).

Written from the general 3-D definitions -- Hamilton products, rotation by r v r*,
translation 2 d r* -- with no planar reduction, so that it checks the oracle's 4-component
planar form rather than restating it.
"""
import numpy as np


def qmul(a, b):
    a0, a1, a2, a3 = a
    b0, b1, b2, b3 = b
    return np.array([a0 * b0 - a1 * b1 - a2 * b2 - a3 * b3,
                     a0 * b1 + a1 * b0 + a2 * b3 - a3 * b2,
                     a0 * b2 - a1 * b3 + a2 * b0 + a3 * b1,
                     a0 * b3 + a1 * b2 - a2 * b1 + a3 * b0])


def conj(a):
    return np.array([a[0], -a[1], -a[2], -a[3]])


def axis_angle(axis, angle):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[np.cos(angle / 2)], np.sin(angle / 2) * axis])


def dq_from_rotation_translation(r, t3):
    """Unit DQ (real, dual) of x -> R x + t."""
    return np.asarray(r, float), 0.5 * qmul(np.concatenate([[0.0], t3]), r)


def dq_transform(real, dual, v3):
    """Apply a (possibly unnormalised) DQ to a 3-D point after DQB normalisation."""
    n = np.linalg.norm(real)
    r = real / n
    d = dual / n
    rot = qmul(qmul(r, np.concatenate([[0.0], v3])), conj(r))
    tr = 2.0 * qmul(d, conj(r))
    return rot[1:] + tr[1:]


def dqb_point(weights, scales, reals, duals, p2):
    """Scale-and-DQ blend at a 2-D point: s_bar * DQB(p), as a 3-vector."""
    w = np.asarray(weights, float)
    sw = w.sum()
    real = (w[:, None] * reals).sum(0) / sw
    dual = (w[:, None] * duals).sum(0) / sw
    s = (w * scales).sum() / sw
    return s * dq_transform(real, dual, np.array([p2[0], p2[1], 0.0]))
