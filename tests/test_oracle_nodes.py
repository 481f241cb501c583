"""Pins of the oracle's node tracking (Eq. 5 with App. A's warp update and Eq. 9's
uncertainty propagation) and EKF merge (Eqs. 12-15)."""
import json
import math
import os

import numpy as np
import pytest

import dq8

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden', 'parameters.json')


def _row(orc, s, th, tx, ty):
    r = np.zeros(8)
    r[:4] = orc.dq_from_rt(th, tx, ty)
    if r[0] < 0:
        r[:4] = -r[:4]
    r[4], r[5] = s, 1.0
    return r


def _apply(orc, row, x):
    q = row[:4] / math.hypot(row[0], row[1])
    return np.array([orc.apply_warp(row[4], q, px, py) for px, py in x])


def test_compose_is_the_composition_of_the_two_warps(orc):
    """App. A's requirement, s_new q_new(x) = ds dq(s_old q_old(x)), checked by applying the
    warps one after the other at random points."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        w_old = _row(orc, rng.uniform(0.8, 1.25), rng.uniform(-0.6, 0.6), *rng.uniform(-40, 40, 2))
        dw = _row(orc, rng.uniform(0.8, 1.25), rng.uniform(-0.6, 0.6), *rng.uniform(-40, 40, 2))
        w_new = orc.compose(w_old, dw)
        x = rng.uniform(-500, 1500, (10, 2))
        np.testing.assert_allclose(_apply(orc, w_new, x), _apply(orc, dw, _apply(orc, w_old, x)),
                                   atol=1e-9)
        assert w_new[0] >= 0 and w_new[4] == pytest.approx(dw[4] * w_old[4])


def test_compose_follows_the_printed_steps_of_appendix_a(orc):
    """App. A's steps with the independent 8-D dual quaternions: q1 = trans2dq((1 - s_old) /
    s_old dt), q2 = dq * q1, q_new = q_old * q2, s_new = ds s_old -- with the product p * q
    read as 'p, then q' (the order under which the steps meet App. A's requirement)."""
    rng = np.random.default_rng(2)

    def dq(th, t):
        return dq8.dq_from_rotation_translation(dq8.axis_angle([0, 0, 1], th), [t[0], t[1], 0.0])

    def then(p, q):            # the DQ of "apply p, then q" = q p in the Hamilton order
        return dq8.qmul(q[0], p[0]), dq8.qmul(q[0], p[1]) + dq8.qmul(q[1], p[0])

    for _ in range(10):
        so, tho, to = rng.uniform(0.8, 1.25), rng.uniform(-0.5, 0.5), rng.uniform(-30, 30, 2)
        ds, dth, dt = rng.uniform(0.8, 1.25), rng.uniform(-0.5, 0.5), rng.uniform(-30, 30, 2)
        q1 = dq(0.0, (1 - so) / so * dt)
        q2 = then(dq(dth, dt), q1)
        qn = then(dq(tho, to), q2)
        want = orc.compose(_row(orc, so, tho, *to), _row(orc, ds, dth, *dt))
        x = rng.uniform(-300, 900, (6, 2))
        got = np.array([ds * so * dq8.dq_transform(qn[0], qn[1], [px, py, 0.0])[:2] for px, py in x])
        np.testing.assert_allclose(got, _apply(orc, want, x), atol=1e-9)


def test_node_track_uniform_field_and_propagation(orc):
    """Every match carrying one similarity dW: each node's warp becomes f(W_old, dW) exactly,
    and its uncertainty ds^2 sigma_old^2 plus Eq. 8 at the node's position at t-1."""
    rng = np.random.default_rng(3)
    n, nn = 60, 25
    src = rng.uniform(0, 640, (n, 2))
    dw = _row(orc, 1.04, 0.03, 6.0, -2.0)
    q8 = np.tile(dw, (n, 1))
    c = np.where(rng.uniform(0, 1, n) < 0.8, 1.0, 0.0)
    x0 = rng.uniform(0, 640, (nn, 2))
    w_old = np.array([_row(orc, rng.uniform(0.9, 1.1), rng.uniform(-0.2, 0.2), *rng.uniform(-20, 20, 2))
                      for _ in range(nn)])
    s2_old = rng.uniform(0.5, 5.0, nn)
    alpha, beta = orc.alpha_for_frame(640, 480), orc.beta_for_frame(640, 480)
    w_new, s2_new = orc.node_track(x0, w_old, s2_old, q8, c, src, alpha, beta)
    for i in range(nn):
        np.testing.assert_allclose(w_new[i], orc.compose(w_old[i], dw), atol=1e-12)
        p = _apply(orc, w_old[i], x0[i:i + 1])
        du = orc.uncertainty_points(c, src, p, beta)[0]
        assert s2_new[i] == pytest.approx(dw[4] ** 2 * s2_old[i] + du, rel=1e-12)
    # no inlier: warps kept, uncertainty infinite
    w2, s22 = orc.node_track(x0, w_old, s2_old, q8, np.zeros(n), src, alpha, beta)
    np.testing.assert_array_equal(w2, w_old)
    assert np.isinf(s22).all()


def test_gamma_is_the_printed_coefficient(orc):
    g = json.load(open(GOLDEN))['gamma']['value']
    assert orc.gamma_for_frame(480, 270) == pytest.approx(g, rel=1e-15)


def _merge_case(orc, rng, nn=30, same=False):
    x0 = rng.uniform(0, 640, (nn, 2))
    mk = lambda: np.array([_row(orc, rng.uniform(0.95, 1.05), rng.uniform(-0.1, 0.1),
                                *rng.uniform(-10, 10, 2)) for _ in range(nn)])
    wt, wl = mk(), mk()
    wk = wt.copy() if same else mk()
    return x0, wt, rng.uniform(0.5, 4, nn), wl, rng.uniform(0.5, 4, nn), wk


def test_merge_against_the_matrix_inverse(orc):
    """Eqs. 12-15 with numpy's inverse of A: merged uncertainty 1/sum(A^-1), weights
    sigma^2 A^-1 [1 1]^T; the merged warp is the weighted average of the two."""
    rng = np.random.default_rng(5)
    x0, wt, vt, wl, vl, wk = _merge_case(orc, rng)
    gamma = orc.gamma_for_frame(640, 480)
    wo, so = orc.node_merge(x0, wt, vt, wl, vl, wk, gamma)
    for i in range(len(vt)):
        d = _apply(orc, wt[i], x0[i:i + 1]) - _apply(orc, wk[i], x0[i:i + 1])
        eta = math.exp(-gamma * float((d ** 2).sum()))
        A = np.array([[vt[i], eta * math.sqrt(vt[i] * vl[i])], [eta * math.sqrt(vt[i] * vl[i]), vl[i]]])
        Ai = np.linalg.inv(A)
        sm = 1.0 / Ai.sum()
        w = sm * Ai @ np.ones(2)
        if (w < 0).any():
            pick = 0 if vt[i] <= vl[i] else 1
            np.testing.assert_array_equal(wo[i], [wt, wl][pick][i])
            assert so[i] == min(vt[i], vl[i])
            continue
        assert so[i] == pytest.approx(sm, rel=1e-10)
        q = w[0] * wt[i, :4] + w[1] * wl[i, :4]
        np.testing.assert_allclose(wo[i, :4], q / math.hypot(q[0], q[1]), atol=1e-12)
        assert wo[i, 4] == pytest.approx(w @ np.array([wt[i, 4], wl[i, 4]]), rel=1e-12)


def test_merge_special_cases(orc):
    rng = np.random.default_rng(6)
    x0, wt, vt, wl, vl, wk = _merge_case(orc, rng)
    # gamma -> infinity: eta = 0, the linear (independent-sensor) merge
    wo, so = orc.node_merge(x0, wt, vt, wl, vl, wk, 1e6)
    np.testing.assert_allclose(so, vt * vl / (vt + vl), rtol=1e-12)
    np.testing.assert_allclose(wo[:, 4], (vl * wt[:, 4] + vt * wl[:, 4]) / (vt + vl), rtol=1e-12)
    # the current frame at its key frame (eta = 1): the estimate with the smaller uncertainty
    x0, wt, vt, wl, vl, wk = _merge_case(orc, rng, same=True)
    wo, so = orc.node_merge(x0, wt, vt, wl, vl, wk, 1e-3)
    np.testing.assert_array_equal(so, np.minimum(vt, vl))
    # equal estimates merge to themselves; the merged uncertainty never exceeds the smaller
    wo, so = orc.node_merge(x0, wt, vt, wt, vt, wk * 0 + _row(orc, 1.0, 0.0, 300.0, 0.0), 1e-3)
    np.testing.assert_allclose(wo, wt, atol=1e-12)
    x0, wt, vt, wl, vl, wk = _merge_case(orc, rng)
    wo, so = orc.node_merge(x0, wt, vt, wl, vl, wk, orc.gamma_for_frame(640, 480))
    assert (so <= np.minimum(vt, vl) * (1 + 1e-12)).all()


def test_node_restrict_against_brute_force_and_limits(orc):
    """Eq. 11: the bound min_j (sigma_j^2 + exp(beta d^2)) by numpy over all pairs; a node on a
    feature is bounded by that feature's uncertainty + 1; no feature leaves sigma^2 unchanged."""
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 640, (50, 2))
    s2 = rng.uniform(1, 400, 50)
    y = rng.uniform(0, 640, (80, 2))
    s2f = rng.uniform(0, 5, 80)
    beta = orc.beta_for_frame(640, 480)
    got = orc.node_restrict(x, s2, y, s2f, beta)
    d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    with np.errstate(over='ignore'):                  # far pairs: exp overflows to +inf
        want = np.minimum(s2, (s2f[None, :] + np.exp(beta * d2)).min(1))
    np.testing.assert_allclose(got, want, rtol=1e-15)
    on = orc.node_restrict(y[:1], np.array([1e9]), y, s2f, beta)
    assert on[0] <= s2f[0] + 1.0
    np.testing.assert_array_equal(orc.node_restrict(x, s2, np.zeros((0, 2)), np.zeros(0), beta), s2)


def test_keyframe_distances(orc):
    """Eq. 6: a key frame equal to the current nodes is at distance 0; a uniform shift by v is at
    |v|; the mean, not the sum or the maximum."""
    rng = np.random.default_rng(12)
    xt = rng.uniform(0, 640, (40, 2))
    xk = np.stack([xt, xt + [3.0, 4.0], xt + np.where(np.arange(40)[:, None] < 20, [6.0, 8.0], [0.0, 0.0])])
    np.testing.assert_allclose(orc.keyframe_distances(xt, xk), [0.0, 5.0, 5.0], atol=1e-12)


def test_feature_uncertainty(orc):
    """Eq. 10: an inlier adds its leave-one-out squared error under the field of the other
    inliers (zero on an exact similarity), an outlier propagates as a node (Eq. 9 at its
    position: ds^2 sigma^2 + Eq. 8)."""
    rng = np.random.default_rng(13)
    n = 120
    src = rng.uniform(0, 640, (n, 2))
    th, s, t = 0.05, 1.04, np.array([7.0, -3.0])
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    dst = s * (src @ R.T + t)
    q8 = np.tile(_row(orc, s, th, *t), (n, 1))
    c = np.where(np.arange(n) % 4 == 0, 0.0, 0.9)
    alpha, beta = orc.alpha_for_frame(640, 480), orc.beta_for_frame(640, 480)
    s2 = rng.uniform(0.5, 3, n)
    got = orc.feature_uncertainty(src, dst, q8, c, alpha, beta, s2)
    inl = c > 0
    np.testing.assert_allclose(got[inl], s2[inl], atol=1e-9)           # exact field: no error
    du = orc.uncertainty_points(c, src, src[~inl], beta)
    np.testing.assert_allclose(got[~inl], s ** 2 * s2[~inl] + du, rtol=1e-12)
    # a displaced inlier adds its squared displacement against the others' (exact) field
    dst2 = dst.copy()
    dst2[1] += [3.0, 4.0]
    got2 = orc.feature_uncertainty(src, dst2, q8, c, alpha, beta, s2)
    assert got2[1] == pytest.approx(s2[1] + 25.0, rel=1e-9)


def _varied_rows(orc, rng, n):
    return np.array([_row(orc, rng.uniform(0.9, 1.1), rng.uniform(-0.15, 0.15), *rng.uniform(-25, 25, 2))
                     for _ in range(n)])


def test_node_track_moves_each_node_with_the_field_at_its_position(orc):
    """Eq. 5 on a field that varies over the image: a node's new warp maps x_0 to where the
    EMDQ field (Eqs. 2-4, evaluated independently at points) takes the node's position at t-1,
    p = W_old(x_0), not its reference position; Eq. 9 uses the field's scale at p."""
    rng = np.random.default_rng(21)
    n, nn = 80, 30
    src = rng.uniform(0, 640, (n, 2))
    q8 = _varied_rows(orc, rng, n)
    c = np.where(rng.uniform(0, 1, n) < 0.8, rng.uniform(0.5, 1.0, n), 0.0)
    x0 = rng.uniform(100, 540, (nn, 2))
    w_old = np.array([_row(orc, rng.uniform(0.95, 1.05), rng.uniform(-0.1, 0.1), *rng.uniform(-60, 60, 2))
                      for _ in range(nn)])
    s2_old = rng.uniform(0.5, 5.0, nn)
    alpha, beta = orc.alpha_for_frame(640, 480), orc.beta_for_frame(640, 480)
    w_new, s2_new = orc.node_track(x0, w_old, s2_old, q8, c, src, alpha, beta)
    for i in range(nn):
        p = _apply(orc, w_old[i], x0[i:i + 1])
        assert np.hypot(*(p[0] - x0[i])) > 5.0                 # the node has moved away from x_0
        want = p + orc.field_points(q8, c, src, p, alpha)
        np.testing.assert_allclose(_apply(orc, w_new[i], x0[i:i + 1]), want, atol=1e-9)
        wgt = c * np.exp(-alpha * ((src - p[0]) ** 2).sum(1))
        ds = (wgt * q8[:, 4]).sum() / wgt.sum()
        du = orc.uncertainty_points(c, src, p, beta)[0]
        assert s2_new[i] == pytest.approx(ds ** 2 * s2_old[i] + du, rel=1e-12)


def test_gamma_scales_with_the_squared_frame_scale(orc):
    """Sec. III-G: gamma is multiplied by 1/s^2, s = (w/480 + h/270)/2; at 960x540 s = 2."""
    g = json.load(open(GOLDEN))['gamma']['value']
    assert orc.gamma_for_frame(960, 540) == pytest.approx(g / 4.0, rel=1e-15)
    assert orc.gamma_for_frame(240, 135) == pytest.approx(g * 4.0, rel=1e-15)


def test_feature_uncertainty_of_an_inlier_on_a_varying_field(orc):
    """Eq. 10's inlier term on a field that varies over the image: the squared distance from
    y_j to where the field of the other matches (Eqs. 2-4 at the point, with match j removed)
    takes x_j."""
    rng = np.random.default_rng(22)
    n = 60
    src = rng.uniform(0, 640, (n, 2))
    q8 = _varied_rows(orc, rng, n)
    c = np.where(np.arange(n) % 5 == 0, 0.0, rng.uniform(0.6, 1.0, n))
    dst = src + rng.normal(0, 4, (n, 2)) + [5.0, -3.0]
    alpha, beta = orc.alpha_for_frame(640, 480), orc.beta_for_frame(640, 480)
    s2 = rng.uniform(0.5, 3, n)
    got = orc.feature_uncertainty(src, dst, q8, c, alpha, beta, s2)
    for j in np.flatnonzero(c > 0)[:12]:
        keep = np.arange(n) != j
        pj = src[j:j + 1]
        yhat = pj + orc.field_points(q8[keep], c[keep], src[keep], pj, alpha)
        assert got[j] == pytest.approx(s2[j] + float(((dst[j] - yhat[0]) ** 2).sum()), rel=1e-9)
