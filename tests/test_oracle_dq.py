"""Pins of the oracle's planar dual-quaternion algebra (Eq. 1 and its footnote)."""
import json
import math
import os

import numpy as np
import pytest

from dq8 import axis_angle, dq_from_rotation_translation, dq_transform

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden', 'parameters.json')


def test_planar_dq_is_the_8d_dq_with_zeros_removed(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        th = rng.uniform(-3.0, 3.0)
        t = rng.uniform(-300, 300, 2)
        real, dual = dq_from_rotation_translation(axis_angle([0, 0, 1], th), [t[0], t[1], 0.0])
        # the footnote's 4 always-zero components
        assert abs(real[1]) < 1e-15 and abs(real[2]) < 1e-15
        assert abs(dual[0]) < 1e-12 and abs(dual[3]) < 1e-12
        q = orc.dq_from_rt(th, t[0], t[1])
        sgn = 1.0 if real[0] >= 0 else -1.0      # antipodal representative
        np.testing.assert_allclose(q, sgn * np.array([real[0], real[3], dual[1], dual[2]]),
                                   rtol=0, atol=1e-12)


def test_dq_round_trip(orc):
    rng = np.random.default_rng(2)
    for _ in range(50):
        th = rng.uniform(-3.1, 3.1)
        t = rng.uniform(-500, 500, 2)
        th2, tx, ty = orc.rt_from_dq(orc.dq_from_rt(th, *t))
        assert abs(th2 - th) < 1e-12
        assert abs(tx - t[0]) < 1e-9 and abs(ty - t[1]) < 1e-9


def test_apply_warp_is_the_similarity_of_eq1(orc):
    """s (R x + t) with R built from the angle as a matrix."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        th, s = rng.uniform(-1, 1), rng.uniform(0.5, 2.0)
        t = rng.uniform(-100, 100, 2)
        p = rng.uniform(-50, 1500, 2)
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        want = s * (R @ p + t)
        got = orc.apply_warp(s, orc.dq_from_rt(th, *t), *p)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-9)
        # also equal to the general 3-D DQ transform of (p, 0)
        real, dual = dq_from_rotation_translation(axis_angle([0, 0, 1], th), [t[0], t[1], 0])
        np.testing.assert_allclose(got, s * dq_transform(real, dual, [p[0], p[1], 0])[:2],
                                   rtol=0, atol=1e-9)


def test_apply_warp_normalises_the_blend(orc):
    q = orc.dq_from_rt(0.4, 10.0, -3.0)
    a = orc.apply_warp(1.1, q, 20.0, 30.0)
    b = orc.apply_warp(1.1, 3.7 * q, 20.0, 30.0)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-10)


def test_alpha_follows_the_resolution_rule(orc):
    g = json.load(open(GOLDEN))
    a0 = g['alpha']['value']
    w0, h0 = g['reference_resolution']['value']
    assert orc.alpha_for_frame(w0, h0) == pytest.approx(a0, rel=1e-15)
    # doubling both dimensions doubles s and quarters alpha
    assert orc.alpha_for_frame(2 * w0, 2 * h0) == pytest.approx(a0 / 4, rel=1e-15)
    # 640x480: s = (4/3 + 16/9)/2 = 14/9
    assert orc.alpha_for_frame(640, 480) == pytest.approx(a0 / (14 / 9) ** 2, rel=1e-14)
