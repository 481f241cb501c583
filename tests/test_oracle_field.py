"""Pins of the oracle's dense field (Eqs. 2-4)."""
import math

import numpy as np

from dq8 import axis_angle, dq_from_rotation_translation, dqb_point


def _rows(orc, s, th, t):
    q = orc.dq_from_rt(th, t[0], t[1])
    return np.array([q[0], q[1], q[2], q[3], s, 1.0, 0.0, 0.0])


def test_identical_transforms_reproduce_the_transform(orc):
    """N copies of one (s, th, t) give exactly that similarity at every pixel."""
    rng = np.random.default_rng(5)
    n = 37
    s, th, t = 1.05, math.radians(5), np.array([12.0, -7.0])
    q8 = np.tile(_rows(orc, s, th, t), (n, 1))
    src = rng.uniform(0, 640, (n, 2))
    c = rng.uniform(0.1, 1.0, n)
    grid = (-8, -5, 70, 40)
    alpha = orc.alpha_for_frame(640, 480)
    d = orc.field(q8, c, src, grid, alpha)
    ys, xs = np.mgrid[grid[1]:grid[1] + grid[3], grid[0]:grid[0] + grid[2]].astype(float)
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    P = np.stack([xs, ys], -1)
    want = s * (P @ R.T + t) - P
    assert np.abs(d - want).max() < 1e-9


def test_brute_force_8d_dq_blend_tiny(orc):
    """N <= 8 on a 16x16 grid against an independent 8-D DQ blend."""
    rng = np.random.default_rng(6)
    for trial in range(4):
        n = int(rng.integers(2, 9))
        src = rng.uniform(0, 16, (n, 2))
        ths = rng.uniform(-0.5, 0.5, n)
        ts = rng.uniform(-20, 20, (n, 2))
        ss = rng.uniform(0.8, 1.25, n)
        c = rng.uniform(0.0, 1.0, n)
        c[0] = 1.0
        q8 = np.stack([_rows(orc, ss[i], ths[i], ts[i]) for i in range(n)])
        reals, duals = zip(*[dq_from_rotation_translation(axis_angle([0, 0, 1], ths[i]),
                                                          [ts[i, 0], ts[i, 1], 0])
                             for i in range(n)])
        reals, duals = np.array(reals), np.array(duals)
        alpha = 0.01
        d = orc.field(q8, c, src, (0, 0, 16, 16), alpha)
        for y in range(16):
            for x in range(16):
                w = c * np.exp(-alpha * ((src - [x, y]) ** 2).sum(1))
                want = dqb_point(w, ss, reals, duals, (x, y))
                assert abs(want[2]) < 1e-9
                np.testing.assert_allclose(d[y, x], want[:2] - [x, y], rtol=0, atol=1e-9)


def test_symmetric_rotations_cancel_at_the_midpoint(orc):
    """Equal weights on rotations +th and -th blend to no rotation; scales average."""
    th = 0.3
    q8 = np.stack([_rows(orc, 1.2, th, [0, 0]), _rows(orc, 0.8, -th, [0, 0])])
    src = np.array([[0.0, 10.0], [20.0, 10.0]])
    d = orc.field_points(q8, np.ones(2), src, np.array([[10.0, 3.0]]), 0.02)
    # blended rotation is 0 and the scale is 1.0: the point stays where it is
    np.testing.assert_allclose(d[0], [0.0, 0.0], atol=1e-12)


def test_field_no_weight_is_nan(orc):
    q8 = np.tile(_rows(orc, 1.0, 0.0, [0, 0]), (3, 1))
    d = orc.field(q8, np.zeros(3), np.zeros((3, 2)), (0, 0, 2, 2), 1e-3)
    assert np.isnan(d).all()


def test_field_permutation_invariant(orc):
    rng = np.random.default_rng(7)
    n = 50
    src = rng.uniform(0, 100, (n, 2))
    q8 = np.stack([_rows(orc, rng.uniform(0.9, 1.1), rng.uniform(-.2, .2),
                         rng.uniform(-5, 5, 2)) for _ in range(n)])
    c = rng.uniform(0, 1, n)
    perm = rng.permutation(n)
    a = orc.field(q8, c, src, (0, 0, 30, 20), 1e-3)
    b = orc.field(q8[perm], c[perm], src[perm], (0, 0, 30, 20), 1e-3)
    assert np.abs(a - b).max() < 1e-10
