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


def test_features_on_a_translation_and_an_outlier():
    """A pure translation: every consistency residual vanishes and the distances are the
    nearest-neighbour distances.  One gross outlier: its residuals against its neighbours
    exceed every inlier's smallest one."""
    g = np.random.default_rng(5)
    x = g.uniform(0, 639, (120, 2))
    y = x + np.array([12.0, -7.0])
    f = ws.features(x, y)
    assert np.abs(f[:, :8]).max() < 1e-9
    from scipy.spatial import cKDTree
    d, _ = cKDTree(np.float32(x).astype(np.float64)).query(np.float32(x).astype(np.float64), k=9)
    np.testing.assert_allclose(f[:, 8:], np.log1p(d[:, 1:]), rtol=0, atol=1e-4)
    y2 = _similarity(x, 1.02, 0.03, np.array([12.0, -7.0]))
    y2[7] += [40.0, 25.0]
    f = ws.features(x, y2)
    others = np.delete(np.arange(120), 7)
    assert f[7, :8].min() > f[others, 0].max()
    assert np.all(np.diff(f[:, :8], axis=1) >= 0) and np.all(np.diff(f[:, 8:], axis=1) >= 0)
    # the distance features are those of the matches in the reference frame (x), whatever
    # the motion: under a scaling by 2 they stay the nearest-neighbour distances of x
    f = ws.features(x, 2.0 * x)
    np.testing.assert_allclose(f[:, 8:], np.log1p(d[:, 1:]), rtol=0, atol=1e-4)
