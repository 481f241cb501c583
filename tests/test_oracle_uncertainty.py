"""Pins of the oracle's EMDQ uncertainty (Eq. 8: the minimum over the feature inliers of
exp(beta d^2)), against an independent nearest-neighbour search (scipy's k-d tree) and the
properties the definition fixes."""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden', 'parameters.json')


def test_beta_is_the_printed_coefficient_scaled_by_the_resolution(orc):
    beta = json.load(open(GOLDEN))['beta']['value']
    assert orc.beta_for_frame(480, 270) == pytest.approx(beta, rel=1e-15)
    s = (1280 / 480 + 1024 / 270) / 2
    assert orc.beta_for_frame(1280, 1024) == pytest.approx(beta / s ** 2, rel=1e-15)


def test_nearest_inlier_by_kd_tree(orc):
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(4)
    n = 300
    src = rng.uniform(0, 640, (n, 2))
    c = np.where(rng.uniform(0, 1, n) < 0.7, rng.uniform(0.5, 1, n), 0.0)
    beta = orc.beta_for_frame(640, 480)
    grid = (-20, -10, 97, 61)
    got = orc.uncertainty(c, src, grid, beta)
    ys, xs = np.mgrid[grid[1]:grid[1] + grid[3], grid[0]:grid[0] + grid[2]]
    d, _ = cKDTree(src[c > 0]).query(np.stack([xs.ravel(), ys.ravel()], 1).astype(np.float64))
    want = np.exp(beta * d ** 2).reshape(grid[3], grid[2])
    np.testing.assert_allclose(got, want, rtol=1e-12)
    pts = rng.uniform(-50, 700, (500, 2))
    d2, _ = cKDTree(src[c > 0]).query(pts)
    np.testing.assert_allclose(orc.uncertainty_points(c, src, pts, beta), np.exp(beta * d2 ** 2),
                               rtol=1e-12)


def test_definition_properties(orc):
    rng = np.random.default_rng(9)
    src = rng.uniform(0, 200, (40, 2))
    src[0] = (50.0, 60.0)
    c = np.ones(40)
    beta = 3e-3
    # 1 exactly at an inlier, above 1 elsewhere
    u = orc.uncertainty(c, src, (50, 60, 1, 1), beta)
    assert u[0, 0] == 1.0
    assert (orc.uncertainty(c, src, (0, 0, 64, 64), beta) >= 1.0).all()
    # outliers (c = 0) are not features: adding them changes nothing
    far = np.vstack([src, rng.uniform(0, 200, (25, 2))])
    cf = np.concatenate([c, np.zeros(25)])
    np.testing.assert_array_equal(orc.uncertainty(cf, far, (0, 0, 64, 64), beta),
                                  orc.uncertainty(c, src, (0, 0, 64, 64), beta))
    # permutation invariance
    perm = rng.permutation(40)
    np.testing.assert_array_equal(orc.uncertainty(c[perm], src[perm], (0, 0, 64, 64), beta),
                                  orc.uncertainty(c, src, (0, 0, 64, 64), beta))
    # increasing along a ray away from a lone inlier
    one = orc.uncertainty(np.array([1.0]), np.array([[0.0, 0.0]]), (0, 0, 50, 1), beta)[0]
    assert (np.diff(one) > 0).all()
    # no inlier: +inf everywhere
    assert np.isinf(orc.uncertainty(np.zeros(40), src, (0, 0, 8, 8), beta)).all()
