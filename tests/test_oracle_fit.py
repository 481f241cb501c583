"""Pins of the oracle's EMDQ fit: M-step (Eqs. 16-20), leave-one-out residuals, EM loop."""
import math

import numpy as np
import pytest
import torch

from dq8 import axis_angle, dq_from_rotation_translation, dqb_point
from synth import make_scene, make_matches, gt_forward


def _similarity(x, s, th, t):
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    return s * (x @ R.T + t)


def test_mstep_exact_on_noise_free_similarity(orc):
    """Every local fit of an exact similarity is that similarity, whatever alpha and p."""
    rng = np.random.default_rng(10)
    s, th, t = 1.05, math.radians(5), np.array([12.0, -7.0])
    x = rng.uniform(0, 640, (120, 2))
    y = _similarity(x, s, th, t)
    for alpha in (1e-5, 8e-5, 1e-3):
        m = orc.mstep(x, y, rng.uniform(0.2, 1.0, 120), alpha)
        assert m['status'] == 0
        assert np.abs(m['s'] - s).max() < 1e-12
        assert np.abs(m['theta'] - th).max() < 1e-12
        assert np.abs(m['t'] - t).max() < 1e-9


def test_mstep_rotation_matches_svd_of_eq18(orc):
    """R = U V^T from svd(C_t C_0^T) (det-corrected), on noisy data with random weights."""
    rng = np.random.default_rng(11)
    n = 60
    x = rng.uniform(0, 300, (n, 2))
    y = _similarity(x, 0.9, 0.7, [5, 9]) + rng.normal(0, 8, (n, 2))
    p = rng.uniform(0.0, 1.0, n)
    alpha = 2e-4
    m = orc.mstep(x, y, p, alpha)
    for i in range(0, n, 7):
        om = p * np.exp(-alpha * ((x - x[i]) ** 2).sum(1))
        xb = (om[:, None] * x).sum(0) / om.sum()
        yb = (om[:, None] * y).sum(0) / om.sum()
        C0 = (np.sqrt(om)[:, None] * (x - xb)).T
        Ct = (np.sqrt(om)[:, None] * (y - yb)).T
        U, _, Vt = np.linalg.svd(Ct @ C0.T)
        D = np.diag([1.0, np.sign(np.linalg.det(U @ Vt))])
        R = U @ D @ Vt
        assert abs(math.atan2(R[1, 0], R[0, 0]) - m['theta'][i]) < 1e-9
        # Eq. 19 norm ratio and Eq. 20: the fitted similarity maps the x-centroid onto the
        # y-centroid
        assert m['s'][i] == pytest.approx(np.linalg.norm(Ct) / np.linalg.norm(C0), rel=1e-12)
        np.testing.assert_allclose(_similarity(xb, m['s'][i], m['theta'][i], m['t'][i]), yb,
                                   atol=1e-9)


def test_mstep_angle_is_the_maximiser(orc):
    rng = np.random.default_rng(12)
    x = rng.uniform(0, 200, (40, 2))
    y = _similarity(x, 1.1, -0.4, [3, 3]) + rng.normal(0, 5, (40, 2))
    p = np.ones(40)
    m = orc.mstep(x, y, p, 5e-4)
    i = 3
    om = np.exp(-5e-4 * ((x - x[i]) ** 2).sum(1))
    xb = (om[:, None] * x).sum(0) / om.sum()
    yb = (om[:, None] * y).sum(0) / om.sum()

    def obj(a):
        R = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
        return (om * (((y - yb) @ R) * (x - xb)).sum(1)).sum()
    grid = np.linspace(-math.pi, math.pi, 20001)
    best = max(obj(a) for a in grid)
    assert obj(m['theta'][i]) >= best - 1e-9 * abs(best)


def test_residuals_brute_force_leave_one_out(orc):
    rng = np.random.default_rng(13)
    n = 6
    x = rng.uniform(0, 30, (n, 2))
    y = x + rng.uniform(-3, 3, (n, 2))
    p = rng.uniform(0.3, 1.0, n)
    ths, ss = rng.uniform(-.3, .3, n), rng.uniform(.9, 1.1, n)
    ts = rng.uniform(-4, 4, (n, 2))
    q8 = np.zeros((n, 8))
    for i in range(n):
        q8[i, :4] = orc.dq_from_rt(ths[i], *ts[i])
        q8[i, 4], q8[i, 5] = ss[i], 1.0
    alpha = 3e-3
    e = orc.residuals(x, y, p, q8, alpha)
    reals, duals = zip(*[dq_from_rotation_translation(axis_angle([0, 0, 1], ths[i]),
                                                      [ts[i, 0], ts[i, 1], 0]) for i in range(n)])
    reals, duals = np.array(reals), np.array(duals)
    for j in range(n):
        keep = np.arange(n) != j
        w = p[keep] * np.exp(-alpha * ((x[keep] - x[j]) ** 2).sum(1))
        yh = dqb_point(w, ss[keep], reals[keep], duals[keep], x[j])[:2]
        assert e[j] == pytest.approx(((y[j] - yh) ** 2).sum(), rel=1e-10, abs=1e-12)


def test_fit_exact_similarity_converges_in_one_iteration(orc):
    rng = np.random.default_rng(14)
    s, th, t = 1.05, math.radians(5), np.array([12.0, -7.0])
    x = rng.uniform(0, 639, (200, 2))
    y = _similarity(x, s, th, t)
    r = orc.fit(x, y, 640, 480)
    assert r['status'] == 0 and r['iters'] == 1
    assert r['sigma2'] == 0.25
    assert (r['p'] > 0.9999).all() and (r['c'] == r['p']).all()
    q = orc.dq_from_rt(th, *t)
    assert np.abs(r['q8'][:, :4] - q).max() < 1e-10
    assert np.abs(r['q8'][:, 4] - s).max() < 1e-12
    # field equals the similarity everywhere
    d = orc.field(r['q8'], r['c'], x, (0, 0, 64, 48), orc.alpha_for_frame(640, 480))
    ys, xs = np.mgrid[0:48, 0:64].astype(float)
    P = np.stack([xs, ys], -1)
    assert np.abs(d - (_similarity(P.reshape(-1, 2), s, th, t).reshape(P.shape) - P)).max() < 1e-9


def test_fit_rejects_a_single_gross_outlier(orc):
    rng = np.random.default_rng(15)
    s, th, t = 0.97, -0.05, np.array([4.0, 6.0])
    x = rng.uniform(0, 639, (150, 2))
    y = _similarity(x, s, th, t)
    y[17] += [60.0, -45.0]
    r = orc.fit(x, y, 640, 480)
    assert r['status'] == 0
    assert r['p'][17] < 1e-6 and r['c'][17] == 0.0
    keep = np.arange(150) != 17
    assert (r['p'][keep] > 0.999).all()
    q = orc.dq_from_rt(th, *t)
    # the outlier's weight is ~0, so every fit (its own included) is the similarity
    assert np.abs(r['q8'][:, :4] - q).max() < 1e-5
    assert np.abs(r['q8'][:, 4] - s).max() < 1e-6


def test_fit_permutation_invariant(orc):
    sc = make_scene(3, 640, 480, 1)
    x, y, _ = make_matches(sc, 1, 200, 0.2, 1.0)
    perm = np.random.default_rng(0).permutation(200)
    a = orc.fit(x, y, 640, 480)
    b = orc.fit(x[perm], y[perm], 640, 480)
    assert a['iters'] == b['iters']
    assert np.abs(a['p'][perm] - b['p']).max() < 1e-9
    assert np.abs(a['q8'][perm] - b['q8']).max() < 1e-7


def _recovery(orc, sc, n, outliers, noise, step=8):
    x, y, inl = make_matches(sc, 1, n, outliers, noise)
    r = orc.fit(x, y, sc.w, sc.h)
    lab = r['c'] > 0
    prec = (lab & inl).sum() / max(1, lab.sum())
    rec = (lab & inl).sum() / inl.sum()
    ys, xs = np.mgrid[0:sc.h:step, 0:sc.w:step].astype(float)
    P = np.stack([xs.ravel(), ys.ravel()], 1)
    d = orc.field_points(r['q8'], r['c'], x, P, orc.alpha_for_frame(sc.w, sc.h))
    gt = gt_forward(sc, torch.from_numpy(P), 1).numpy() - P
    err = np.sqrt(((d - gt) ** 2).sum(1))
    inner = (P[:, 0] > 64) & (P[:, 0] < sc.w - 64) & (P[:, 1] > 64) & (P[:, 1] < sc.h - 64)
    return r, prec, rec, err, inner


def test_fit_recovers_a_noisy_similarity_with_outliers(orc):
    """No bumps: 1 px noise, 20% uniform outliers. sigma^2 estimates the per-axis noise
    variance, gamma the inlier fraction, and the field the similarity."""
    sc = make_scene(21, 640, 480, 1, bump_amp=0.0)
    r, prec, rec, err, _ = _recovery(orc, sc, 200, 0.2, 1.0)
    assert r['status'] == 0
    assert prec >= 0.97 and rec >= 0.97
    assert 0.75 <= r['sigma2'] <= 1.3
    assert abs(r['gamma'] - 0.8) < 0.04
    assert np.sqrt((err ** 2).mean()) < 0.35


def test_fit_recovers_the_bumped_field(orc):
    """The 640x480 pair: similarity + 3 bumps (8 px, sigma 60), 20% outliers."""
    sc = make_scene(1, 640, 480, 1)
    r, prec, rec, err, inner = _recovery(orc, sc, 200, 0.2, 1.0)
    assert r['status'] == 0
    assert prec >= 0.95 and rec >= 0.95
    assert np.sqrt((err[inner] ** 2).mean()) < 2.5


def test_fit_iteration_cap_and_bad_input(orc):
    sc = make_scene(1, 640, 480, 1)
    x, y, _ = make_matches(sc, 1, 200, 0.2, 1.0)
    r = orc.fit(x, y, 640, 480, max_iters=2)
    assert r['status'] == 3 and r['iters'] == 2          # ENOCONV, outputs still valid
    assert np.isfinite(r['q8']).all()
    r = orc.fit(x, y, 640, 480, max_iters=4, tol_p=0.0)  # tol 0: always the full count
    assert r['iters'] == 4 and r['status'] == 3
    assert orc.fit(x[:2], y[:2], 640, 480)['status'] == 1   # EINVAL, n < 3


def test_first_posterior_is_the_gaussian_uniform_mixture(orc):
    """One EM iteration: the posterior of each match under a 2-D isotropic Gaussian inlier
    density (scipy) against a uniform outlier density over the frame, with the step-0
    residuals, sigma^2 and the initial mixing weight 1/2 (with warm-start weights p0: step 0
    weighted by p0 and the mixing weight the mean of p0)."""
    from scipy.stats import multivariate_normal
    sc = make_scene(4, 640, 480, 1)
    x, y, _ = make_matches(sc, 1, 120, 0.25, 1.0)
    alpha = orc.alpha_for_frame(640, 480)
    p1 = np.ones(120)
    m = orc.mstep(x, y, p1, alpha)
    e0 = orc.residuals(x, y, p1, m['q8'], alpha)
    s2 = max(e0.sum() / (2 * 120), 0.25)
    r = orc.fit(x, y, 640, 480, max_iters=1)
    # residual vectors: only their length enters an isotropic density
    g = multivariate_normal(mean=[0, 0], cov=s2 * np.eye(2)).pdf(
        np.stack([np.sqrt(e0), np.zeros(120)], 1))
    want = 0.5 * g / (0.5 * g + 0.5 / (640 * 480))
    np.testing.assert_allclose(r['p'], want, rtol=1e-10, atol=1e-300)
    assert r['dp_trace'][0] == pytest.approx(np.abs(want - 1).max(), rel=1e-10)
    # inlier weights of the output: the matches with posterior >= 1/2 keep it, others 0
    np.testing.assert_array_equal(r['c'], np.where(r['p'] >= 0.5, r['p'], 0.0))
    # with warm-start weights p0: step 0 weighted by p0, the mixing weight its mean
    p0 = np.random.default_rng(8).uniform(0.2, 1.0, 120)
    m = orc.mstep(x, y, p0, alpha)
    e0 = orc.residuals(x, y, p0, m['q8'], alpha)
    s2 = max((p0 * e0).sum() / (2 * p0.sum()), 0.25)
    gam = min(max(p0.mean(), 0.05), 0.95)
    r = orc.fit(x, y, 640, 480, max_iters=1, p0=p0)
    g = multivariate_normal(mean=[0, 0], cov=s2 * np.eye(2)).pdf(
        np.stack([np.sqrt(e0), np.zeros(120)], 1))
    want = gam * g / (gam * g + (1 - gam) / (640 * 480))
    np.testing.assert_allclose(r['p'], want, rtol=1e-10, atol=1e-300)
