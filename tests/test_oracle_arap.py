"""Pins of the oracle's ARAP smoothing of node warps (Sec. III-D, Eqs. 21-22)."""
import math

import numpy as np
import pytest


def _row(orc, s, th, tx, ty):
    r = np.zeros(8)
    r[:4] = orc.dq_from_rt(th, tx, ty)
    r[4], r[5] = s, 1.0
    return r


def _pos(orc, w, x0):
    return np.array([orc.apply_warp(r[4], r[:4] / math.hypot(r[0], r[1]), x[0], x[1])
                     for r, x in zip(w, x0)])


def _lattice(step=40.0, w=640, h=480):
    xs, ys = np.meshgrid(np.arange(0, w, step), np.arange(0, h, step))
    return np.stack([xs.ravel(), ys.ravel()], 1).astype(np.float64)


def test_a_common_similarity_is_a_fixed_point(orc):
    x0 = _lattice()
    S = _row(orc, 1.05, 0.08, 12.0, -7.0)
    w = np.tile(S, (len(x0), 1))
    out, costs = orc.arap_smooth(x0, w, np.ones(len(x0)), orc.alpha_for_frame(640, 480))
    np.testing.assert_allclose(_pos(orc, out, x0), _pos(orc, w, x0), atol=1e-8)
    assert costs[0] == pytest.approx(0.0, abs=1e-12)


def test_no_iteration_returns_the_merged_warps(orc):
    x0 = _lattice()
    rng = np.random.default_rng(0)
    w = np.array([_row(orc, 1.0, 0.0, *rng.normal(0, 3, 2)) for _ in x0])
    out, _ = orc.arap_smooth(x0, w, np.ones(len(x0)), 1e-4, max_iters=0)
    np.testing.assert_array_equal(out, w)


def _hand_three_nodes():
    """Eqs. 16-17 and ARAP1-3 worked by hand on three nodes x_0 = (0,0), (1,0), (0,1) that move
    to x_t = (0,0), (2,0), (0,1) (a stretch along x), alpha = ln 2, so a node at distance 1
    weighs 1/2 and one at distance sqrt(2) weighs 1/4.

    Node 0: columns of C_0 (1/2, 0), (0, 1/2) and of C_t (1, 0), (0, 1/2) (its own column is
    zero); C_t C_0^T = [[1/2, 0], [0, 1/4]], angle atan2(0, 3/4) = 0; s = sqrt(5/4) / sqrt(1/2)
    = sqrt(5/2); t = [1 (0,0) + 1/2 (2/s - 1, 0) + 1/2 (0, 1/s - 1)] / 2.
    Node 1: C_0 (-1/2, 0), (-1/4, 1/4); C_t (-1, 0), (-1/2, 1/4); C_t C_0^T = [[5/8, -1/8],
    [-1/16, 1/16]], angle atan2(1/16, 11/16); s = sqrt(21/16) / sqrt(6/16) = sqrt(7/2);
    t = [1/2 (0,0) + 1 (2/s - c, -sn) + 1/4 (sn, 1/s - c)] / (7/4).
    Node 2: C_0 (0, -1/2), (1/4, -1/4); C_t (0, -1/2), (1/2, -1/4); C_t C_0^T = [[1/8, -1/8],
    [-1/16, 5/16]], angle atan2(1/16, 7/16); s = sqrt(9/16) / sqrt(6/16) = sqrt(3/2);
    t = [1/2 (0,0) + 1/4 (2/s - c, -sn) + 1 (sn, 1/s - c)] / (7/4)."""
    out = []
    s0 = math.sqrt(2.5)
    out.append((s0, 0.0, ((2 / s0 - 1) / 4, (1 / s0 - 1) / 4)))
    s1, a1 = math.sqrt(3.5), math.atan2(1.0, 11.0)
    c, sn = math.cos(a1), math.sin(a1)
    out.append((s1, a1, ((2 / s1 - c + sn / 4) / 1.75, (-sn + (1 / s1 - c) / 4) / 1.75)))
    s2, a2 = math.sqrt(1.5), math.atan2(1.0, 7.0)
    c, sn = math.cos(a2), math.sin(a2)
    out.append((s2, a2, (((2 / s2 - c) / 4 + sn) / 1.75, (-sn / 4 + 1 / s2 - c) / 1.75)))
    return out


def test_arap_fit_worked_by_hand_on_three_nodes(orc):
    """Sec. III-D as printed: node-centred columns with the weight inside each column (so C_t
    C_0^T carries w^2), the scale as the norm ratio of those columns, the translation the
    w-weighted average of x_t / s - R x_0.  Against values derived by hand."""
    x0 = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    xt = np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 1.0]])
    got = orc.arap_fit(x0, xt, math.log(2.0))
    assert got['status'] == 0
    for i, (s, a, t) in enumerate(_hand_three_nodes()):
        assert got['s'][i] == pytest.approx(s, abs=1e-13)
        assert got['theta'][i] == pytest.approx(a, abs=1e-13)
        np.testing.assert_allclose(got['t'][i], t, atol=1e-13)
        np.testing.assert_allclose(got['q8'][i, :4], orc.dq_from_rt(a, *t), atol=1e-13)
        assert got['q8'][i, 4] == pytest.approx(s, abs=1e-13)
    # the centroid-centred, weight-once fit of the EM M-step differs on this case
    m = orc.mstep(x0, xt, np.ones(3), math.log(2.0))
    assert np.abs(m['theta'] - got['theta']).max() > 1e-2
    assert np.abs(m['s'] - got['s']).max() > 1e-2


def test_arap_fit_translation_is_the_weighted_average(orc):
    """ARAP3 with the printed R and s: on random motion the translation equals the
    exp(-alpha d^2)-weighted mean of x_t / s - R x_0 (every node j, itself with weight 1), and
    R, s are invariant to a common shift of x_t (node-centred columns), which moves t by the
    shift / s."""
    rng = np.random.default_rng(7)
    x0 = rng.uniform(0, 300, (12, 2))
    xt = x0 + rng.normal(0, 4, (12, 2))
    alpha = 1e-4
    a = orc.arap_fit(x0, xt, alpha)
    shift = np.array([13.0, -5.0])
    b = orc.arap_fit(x0, xt + shift, alpha)
    np.testing.assert_allclose(b['theta'], a['theta'], atol=1e-12)
    np.testing.assert_allclose(b['s'], a['s'], rtol=1e-12)
    np.testing.assert_allclose(b['t'], a['t'] + shift / a['s'][:, None], atol=1e-9)
    for i in range(12):
        w = np.exp(-alpha * ((x0 - x0[i]) ** 2).sum(1))
        R = np.array([[math.cos(a['theta'][i]), -math.sin(a['theta'][i])],
                      [math.sin(a['theta'][i]), math.cos(a['theta'][i])]])
        v = xt / a['s'][i] - x0 @ R.T
        np.testing.assert_allclose(a['t'][i], (w[:, None] * v).sum(0) / w.sum(), atol=1e-9)


def test_arap_fit_rotation_from_the_svd(orc):
    """ARAP1 via numpy's SVD on a rotated, anisotropically stretched lattice: R = U V^T of the
    2 x 2 matrix (det > 0 here, so no reflection fix is involved) has the oracle's angle for
    every node."""
    x0 = _lattice(50.0, 300, 250)
    th = 0.3
    R0 = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    xt = (x0 * [1.2, 0.9]) @ R0.T + [5.0, 2.0]
    alpha = 2e-4
    got = orc.arap_fit(x0, xt, alpha)
    for i in range(0, len(x0), 7):
        w = np.exp(-alpha * ((x0 - x0[i]) ** 2).sum(1))
        C0 = (w[:, None] * (x0 - x0[i])).T
        Ct = (w[:, None] * (xt - xt[i])).T
        U, _, Vt = np.linalg.svd(Ct @ C0.T)
        assert np.linalg.det(U @ Vt) > 0
        R = U @ Vt
        assert math.atan2(R[1, 0], R[0, 0]) == pytest.approx(got['theta'][i], abs=1e-12)
        assert got['s'][i] == pytest.approx(np.linalg.norm(Ct) / np.linalg.norm(C0), rel=1e-12)


def test_first_iteration_is_eq22_with_the_neighbourhood_fit(orc):
    """One iteration: lambda = (1 + sigma^2)/101 weights the ARAP warp, which is the ARAP fit
    (Eqs. 16-17, ARAP1-3) of the nodes' motion x_0 -> W_merge(x_0)."""
    x0 = _lattice()
    rng = np.random.default_rng(1)
    w = np.array([_row(orc, rng.uniform(0.98, 1.02), rng.normal(0, 0.02), *rng.normal(0, 3, 2)) for _ in x0])
    s2 = np.full(len(x0), 100.0)                          # lambda = 1: the plain average
    alpha = orc.alpha_for_frame(640, 480)
    out, _ = orc.arap_smooth(x0, w, s2, alpha, max_iters=1)
    fit = orc.arap_fit(x0, _pos(orc, w, x0), alpha)['q8']
    q = w[:, :4] / np.hypot(w[:, 0], w[:, 1])[:, None] + fit[:, :4] / np.hypot(fit[:, 0], fit[:, 1])[:, None]
    np.testing.assert_allclose(out[:, :4], q / np.hypot(q[:, 0], q[:, 1])[:, None], atol=1e-12)
    np.testing.assert_allclose(out[:, 4], 0.5 * (w[:, 4] + fit[:, 4]), atol=1e-12)


def test_costs_never_increase_and_noise_is_smoothed(orc):
    """A smooth similarity plus independent per-node jitter: the iterations' costs do not
    increase up to the stop, and the smoothed nodes lie closer to the smooth motion."""
    x0 = _lattice(30.0)
    rng = np.random.default_rng(2)
    S = _row(orc, 1.03, 0.05, 8.0, 4.0)
    w = np.array([_row(orc, 1.03 * rng.uniform(0.99, 1.01), 0.05 + rng.normal(0, 0.01), 8.0 + rng.normal(0, 2),
                       4.0 + rng.normal(0, 2)) for _ in x0])
    s2 = rng.uniform(1, 50, len(x0))
    out, costs = orc.arap_smooth(x0, w, s2, orc.alpha_for_frame(640, 480))
    ran = costs[~np.isnan(costs)]
    kept = ran if len(ran) < 2 or ran[-1] <= ran[-2] else ran[:-1]
    assert (np.diff(kept) <= 1e-9 * kept[0]).all()
    truth = _pos(orc, np.tile(S, (len(x0), 1)), x0)
    before = np.abs(_pos(orc, w, x0) - truth).mean()
    after = np.abs(_pos(orc, out, x0) - truth).mean()
    assert after < 0.9 * before


def test_hex_lattice_definition(orc):
    """Sec. III-E: the lattice holds the centre, every node has its 6 neighbours at the spacing
    unless it is near the frame edge, and it covers the frame: no pixel is farther than the
    lattice's covering radius spacing/sqrt(3) from a node."""
    from scipy.spatial import cKDTree
    x = orc.hex_nodes(640, 480, 40.0)
    assert np.any(np.all(np.isclose(x, [319.5, 239.5]), axis=1))
    t = cKDTree(x)
    d, _ = t.query(x, k=7)
    inner = (x[:, 0] > 45) & (x[:, 0] < 594) & (x[:, 1] > 45) & (x[:, 1] < 434)
    np.testing.assert_allclose(d[inner, 1:], 40.0, rtol=1e-9)
    g = np.stack(np.meshgrid(np.arange(0, 640, 7.0), np.arange(0, 480, 7.0)), -1).reshape(-1, 2)
    dg, _ = t.query(g)
    assert dg.max() <= 40.0 / math.sqrt(3.0) + 1e-9


def test_new_node_warps_are_the_weighted_average(orc):
    x0 = _lattice()
    S = _row(orc, 1.05, 0.08, 12.0, -7.0)
    w = np.tile(S, (len(x0), 1))
    pts = np.array([[10.0, 10.0], [333.3, 111.1], [700.0, 500.0]])
    out = orc.node_init(x0, w, pts, orc.alpha_for_frame(640, 480))
    np.testing.assert_allclose(out, np.tile(S, (3, 1)) * [1, 1, 1, 1, 1, 1, 0, 0] + [0] * 8, atol=1e-12)
    # two nodes: the new node midway takes the plain average of their warps
    a, b = _row(orc, 1.0, 0.0, 0.0, 0.0), _row(orc, 1.1, 0.2, 10.0, 0.0)
    mid = orc.node_init(np.array([[0.0, 0.0], [20.0, 0.0]]), np.stack([a, b]), np.array([[10.0, 0.0]]), 1e-3)[0]
    q = a[:4] / math.hypot(a[0], a[1]) + b[:4] / math.hypot(b[0], b[1])
    np.testing.assert_allclose(mid[:4], q / math.hypot(q[0], q[1]), atol=1e-12)
    assert mid[4] == pytest.approx(1.05)


def _jittered(orc, x0, rng):
    return np.array([_row(orc, rng.uniform(0.97, 1.03), rng.normal(0.03, 0.03), *rng.normal([6.0, -4.0], 3))
                     for _ in x0])


def _average(wa, a, wb, b):
    """Eq. 22's weighted average of two rows: the unit DQs and the scales with weights a, b."""
    a = np.broadcast_to(np.asarray(a, float), (len(wa),))
    b = np.broadcast_to(np.asarray(b, float), (len(wa),))
    q = a[:, None] * wa[:, :4] / np.hypot(wa[:, 0], wa[:, 1])[:, None] + b[:, None] * wb[:, :4] / np.hypot(wb[:, 0], wb[:, 1])[:, None]
    return q / np.hypot(q[:, 0], q[:, 1])[:, None], (a * wa[:, 4] + b * wb[:, 4]) / (a + b)


def test_iterations_follow_eq22_and_eq21_with_per_node_lambda(orc):
    """Per-node lambda = (1 + sigma^2)/101 away from 1: iteration 1 averages W_merge (weight 1)
    with the ARAP fit of x_0 -> W_merge(x_0) (weight lambda); its Eq. 21 cost is
    sum |W_merge(x_0) - W^1(x_0)|^2 + lambda |W_ARAP(x_0) - W^1(x_0)|^2; iteration 2 fits
    x_0 -> W^1(x_0), the positions of the first iteration's warps, again averages with W_merge,
    and is kept only if its cost does not rise."""
    x0 = _lattice(35.0)
    rng = np.random.default_rng(3)
    w = _jittered(orc, x0, rng)
    s2 = rng.uniform(0.0, 400.0, len(x0))
    lam = (1.0 + s2) / 101.0
    alpha = orc.alpha_for_frame(640, 480)
    ones = np.ones(len(x0))
    w1, c1 = orc.arap_smooth(x0, w, s2, alpha, max_iters=1)
    fit1 = orc.arap_fit(x0, _pos(orc, w, x0), alpha)['q8']
    q, s = _average(w, ones, fit1, lam)
    np.testing.assert_allclose(w1[:, :4], q, atol=1e-12)
    np.testing.assert_allclose(w1[:, 4], s, atol=1e-12)
    p1, pm, pa = _pos(orc, w1, x0), _pos(orc, w, x0), _pos(orc, fit1, x0)
    cost = (((pm - p1) ** 2).sum(1) + lam * ((pa - p1) ** 2).sum(1)).sum()
    assert c1[0] == pytest.approx(cost, rel=1e-9)
    w2, c2 = orc.arap_smooth(x0, w, s2, alpha, max_iters=2)
    fit2 = orc.arap_fit(x0, p1, alpha)['q8']
    q, s = _average(w, ones, fit2, lam)
    cand = np.concatenate([q, s[:, None], np.tile([1.0, 0.0, 0.0], (len(s), 1))], 1)
    pc, pa2 = _pos(orc, cand, x0), _pos(orc, fit2, x0)
    cost2 = (((pm - pc) ** 2).sum(1) + lam * ((pa2 - pc) ** 2).sum(1)).sum()
    assert c2[1] == pytest.approx(cost2, rel=1e-9)
    if c2[1] > c2[0]:                                       # the cost rose: W^1 is kept
        np.testing.assert_array_equal(w2, w1)
    else:
        np.testing.assert_allclose(w2, cand, atol=1e-12)


def test_new_node_warp_moves_it_with_the_node_field(orc):
    """Sec. III-E on warps that vary over the nodes: a new node at p takes the blend of the
    node warps with weights exp(-alpha |p - x0_j|^2), so its warp maps p where the dense field
    of the nodes (Eqs. 2-4 at the point, every node weight 1) does."""
    x0 = _lattice(45.0)
    rng = np.random.default_rng(4)
    w = _jittered(orc, x0, rng)
    alpha = orc.alpha_for_frame(640, 480)
    pts = rng.uniform(-30, 670, (15, 2))
    out = orc.node_init(x0, w, pts, alpha)
    want = pts + orc.field_points(w, np.ones(len(x0)), x0, pts, alpha)
    np.testing.assert_allclose(_pos(orc, out, pts), want, atol=1e-9)


@pytest.mark.parametrize('w,h,spacing', [(640, 480, 40.0), (1280, 1024, 30.0), (1920, 1080, 55.0),
                                         (500, 333, 37.0), (101, 77, 13.0), (257, 911, 21.5)])
def test_hex_lattice_covers_every_frame_pixel(orc, w, h, spacing):
    """Coverage at several frame sizes and spacings, the corners included: every pixel of the
    frame is within the covering radius spacing/sqrt(3) of a node, and no node lies farther
    than that radius from the frame."""
    from scipy.spatial import cKDTree
    x = orc.hex_nodes(w, h, spacing)
    m = spacing / math.sqrt(3.0)
    gx = np.unique(np.concatenate([np.arange(0, w, 3.0), [w - 1.0]]))
    gy = np.unique(np.concatenate([np.arange(0, h, 3.0), [h - 1.0]]))
    g = np.stack(np.meshgrid(gx, gy), -1).reshape(-1, 2)
    d, _ = cKDTree(x).query(g)
    assert d.max() <= m + 1e-9
    ex = np.maximum(np.maximum(-x[:, 0], 0.0), x[:, 0] - (w - 1))
    ey = np.maximum(np.maximum(-x[:, 1], 0.0), x[:, 1] - (h - 1))
    assert (np.hypot(ex, ey) <= m + 1e-9).all()
