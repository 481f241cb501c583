"""Pins of the FP64 oracle of the learned EM warm start (features, network, loss, Adam)."""
import math

import numpy as np
import pytest

from oracle import warmstart as ws


def _rand_params(seed=0):
    g = np.random.default_rng(seed)
    return g.normal(0, 0.3, ws.N_PARAMS)


def test_parameter_layout():
    assert ws.N_PARAMS == 16 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 5313
    w = _rand_params(1)
    np.testing.assert_array_equal(ws.pack(*ws.unpack(w)), w)


def test_loss_is_the_cross_entropy():
    g = np.random.default_rng(2)
    w = _rand_params(2)
    X = g.normal(0, 1, (50, 16))
    y = (g.uniform(size=50) < 0.4).astype(float)
    p, _ = ws.forward(w, X)
    direct = -np.mean(y * np.log(p) + (1 - y) * np.log(1 - p))
    assert ws.loss(w, X, y) == pytest.approx(direct, rel=1e-12)


def test_gradient_matches_central_differences():
    g = np.random.default_rng(3)
    w = _rand_params(3)
    X = g.normal(0, 1, (40, 16))
    y = (g.uniform(size=40) < 0.5).astype(float)
    an = ws.grad(w, X, y)
    idx = g.choice(ws.N_PARAMS, 200, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(w)
        e[i] = h
        fd = (ws.loss(w + e, X, y) - ws.loss(w - e, X, y)) / (2 * h)
        assert an[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_adam_first_step_is_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    w = np.zeros(4)
    w1, m, v = ws.adam_step(w, g, np.zeros(4), np.zeros(4), t=1, lr=0.01)
    np.testing.assert_allclose(w1, -0.01 * np.sign(g), rtol=1e-4)
    # constant gradients keep the step at lr (bias correction)
    w2, m, v = ws.adam_step(w1, g, m, v, t=2, lr=0.01)
    np.testing.assert_allclose(w2 - w1, -0.01 * np.sign(g), rtol=1e-4)


def test_knn_against_kdtree_and_ties():
    from scipy.spatial import cKDTree
    g = np.random.default_rng(4)
    x = g.uniform(0, 500, (300, 2)).astype(np.float32)
    nn = ws.knn(x)
    d, i = cKDTree(x.astype(np.float64)).query(x.astype(np.float64), k=9)
    for j in range(300):
        assert set(nn[j]) == set(i[j, 1:])
    # equal distances: lower index first
    grid = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [5, 5], [6, 5], [5, 6], [7, 7],
                     [9, 9]], np.float32)
    assert list(ws.knn(grid)[0][:4]) == [1, 2, 3, 4]


def _similarity(x, s, th, t):
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    return s * (x @ R.T + t)


def test_features_vanish_on_an_exact_similarity_and_flag_an_outlier(orc):
    g = np.random.default_rng(5)
    x = g.uniform(0, 639, (120, 2))
    y = _similarity(x, 1.05, 0.08, np.array([12.0, -7.0]))
    m = orc.mstep(x, y, np.ones(120), orc.alpha_for_frame(640, 480))
    f = ws.features(x, y, m['q8'], 1.0)
    assert np.abs(f).max() < 1e-9
    y2 = y.copy()
    y2[7] += [40.0, 25.0]
    m = orc.mstep(x, y2, np.ones(120), orc.alpha_for_frame(640, 480))
    f = ws.features(x, y2, m['q8'], 1.0)
    # the outlier's residual under its neighbours' warps exceeds every inlier's
    others = np.delete(np.arange(120), 7)
    assert f[7, 8:].min() > f[others, 8:].max()
    assert np.all(np.diff(f[:, :8], axis=1) >= 0) and np.all(np.diff(f[:, 8:], axis=1) >= 0)
