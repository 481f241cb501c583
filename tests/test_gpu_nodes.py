"""GPU parity: node tracking (Eq. 5, App. A, Eq. 9) and the EKF merge (Eqs. 12-15) against
the FP64 oracle, on a grid of nodes over frames of the 1280x1024 sequence (fits from the
oracle) and on the merge's special cases."""
import math

import numpy as np
import pytest
import torch

from synth import make_matches, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _f32(a):
    return np.float32(a).astype(np.float64)


def _row(orc, s, th, tx, ty):
    r = np.zeros(8)
    r[:4] = orc.dq_from_rt(th, tx, ty)
    r[4], r[5] = s, 1.0
    return r


def _positions(orc, w, x0):
    out = []
    for row, x in zip(w, x0):
        q = row[:4] / math.hypot(row[0], row[1])
        out.append(orc.apply_warp(row[4], q, x[0], x[1]))
    return np.array(out)


def _nodes(orc, rng, w, h, step=30.0):
    xs, ys = np.meshgrid(np.arange(0, w, step), np.arange(0, h, step))
    x0 = np.stack([xs.ravel(), ys.ravel()], 1)
    x0[::2] += step / 2 * np.array([1.0, 0.0])          # a hexagonal-ish lattice
    nn = x0.shape[0]
    w_old = np.array([_row(orc, rng.uniform(0.97, 1.03), rng.uniform(-0.05, 0.05), *rng.uniform(-8, 8, 2))
                      for _ in range(nn)])
    return x0, w_old, rng.uniform(0.5, 3.0, nn)


def test_node_track_against_the_oracle(emdq, orc):
    sc, cfg = workload('seq1280', seed=4)
    s, d, _ = make_matches(sc, 3, cfg['n'], cfg['outliers'], cfg['noise'])
    fit = orc.fit(_f32(s), _f32(d), sc.w, sc.h)
    rng = np.random.default_rng(8)
    x0, w_old, s2_old = _nodes(orc, rng, sc.w, sc.h)
    alpha, beta = orc.alpha_for_frame(sc.w, sc.h), orc.beta_for_frame(sc.w, sc.h)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    q8 = fit['q8'].astype(np.float32)
    c = fit['c'].astype(np.float32)
    w_new, s2_new = emdq.node_track(f(x0), f(w_old), f(s2_old), f(q8), f(c), f(s),
                                    np.float32(alpha), np.float32(beta))
    torch.cuda.synchronize()
    want_w, want_s2 = orc.node_track(_f32(x0), _f32(w_old), _f32(s2_old), _f32(q8), _f32(c), _f32(s),
                                     float(np.float32(alpha)), float(np.float32(beta)))
    got_w = w_new.cpu().numpy().astype(np.float64)
    # where each node lands at t (the warp's meaning), and its scale and uncertainty
    dpos = np.abs(_positions(orc, got_w, _f32(x0)) - _positions(orc, want_w, _f32(x0))).max()
    print(f'{len(x0)} nodes: max position difference {dpos:.2e} px')
    assert dpos <= 2e-3
    np.testing.assert_allclose(got_w[:, 4], want_w[:, 4], rtol=1e-5)
    assert (got_w[:, 0] >= 0).all()
    np.testing.assert_allclose(s2_new.cpu().numpy(), want_s2, rtol=1e-4)
    # no inlier: warps kept, uncertainty +inf
    w2, s22 = emdq.node_track(f(x0), f(w_old), f(s2_old), f(q8), f(np.zeros_like(c)), f(s),
                              np.float32(alpha), np.float32(beta))
    assert torch.equal(w2, f(w_old)) and torch.isinf(s22).all()


@pytest.mark.parametrize('case', ['general', 'linear', 'at_key_frame'])
def test_node_merge_against_the_oracle(emdq, orc, case):
    rng = np.random.default_rng({'general': 1, 'linear': 2, 'at_key_frame': 3}[case])
    nn = 777
    x0 = rng.uniform(0, 1280, (nn, 2))
    mk = lambda: np.array([_row(orc, rng.uniform(0.95, 1.05), rng.uniform(-0.1, 0.1),
                                *rng.uniform(-6, 6, 2)) for _ in range(nn)])
    wt, wl = mk(), mk()
    wk = wt.copy() if case == 'at_key_frame' else mk()
    vt, vl = rng.uniform(0.5, 4, nn), rng.uniform(0.5, 4, nn)
    gamma = {'general': orc.gamma_for_frame(1280, 1024), 'linear': 1e6, 'at_key_frame': 1e-3}[case]
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    wo, so = emdq.node_merge(f(x0), f(wt), f(vt), f(wl), f(vl), f(wk), np.float32(gamma))
    torch.cuda.synchronize()
    want_w, want_s = orc.node_merge(_f32(x0), _f32(wt), _f32(vt), _f32(wl), _f32(vl), _f32(wk),
                                    float(np.float32(gamma)))
    got_w = wo.cpu().numpy().astype(np.float64)
    dpos = np.abs(_positions(orc, got_w, _f32(x0)) - _positions(orc, want_w, _f32(x0))).max()
    assert dpos <= 1e-3
    np.testing.assert_allclose(so.cpu().numpy(), want_s, rtol=1e-4)
    if case == 'at_key_frame':
        np.testing.assert_array_equal(so.cpu().numpy(), np.float32(np.minimum(vt, vl)))


def test_node_argument_errors(emdq):
    z = torch.zeros((4, 2), device='cuda')
    w = torch.zeros((4, 8), device='cuda')
    v = torch.ones(4, device='cuda')
    with pytest.raises(emdq.EmdqError):
        emdq.node_track(z, w, v, w, v, z, 0.0, 1e-3)
    with pytest.raises(emdq.EmdqError):
        emdq.node_merge(z, w, v, w, v, w, -1.0)


def test_node_restrict_and_keyframe_distances(emdq, orc):
    rng = np.random.default_rng(21)
    x = rng.uniform(0, 1280, (1500, 2))
    s2 = rng.uniform(1, 500, 1500)
    y = rng.uniform(0, 1280, (700, 2))
    s2f = rng.uniform(0, 5, 700)
    beta = orc.beta_for_frame(1280, 1024)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    got = emdq.node_restrict(f(x), f(s2), f(y), f(s2f), np.float32(beta))
    want = orc.node_restrict(_f32(x), _f32(s2), _f32(y), _f32(s2f), float(np.float32(beta)))
    np.testing.assert_allclose(got.cpu().numpy(), want, rtol=1e-5)
    xk = np.stack([x + rng.normal(0, 5 * k, x.shape) for k in range(6)])
    d = emdq.keyframe_distances(f(x), f(xk))
    np.testing.assert_allclose(d.cpu().numpy(), orc.keyframe_distances(_f32(x), _f32(xk)), rtol=1e-5, atol=1e-5)


def test_feature_uncertainty_against_the_oracle(emdq, orc):
    sc, cfg = workload('seq1280', seed=6)
    s, d, _ = make_matches(sc, 2, cfg['n'], cfg['outliers'], cfg['noise'])
    fit = orc.fit(_f32(s), _f32(d), sc.w, sc.h)
    q8, c = fit['q8'].astype(np.float32), fit['c'].astype(np.float32)
    rng = np.random.default_rng(23)
    s2 = rng.uniform(0.5, 3, len(c)).astype(np.float32)
    alpha, beta = np.float32(orc.alpha_for_frame(sc.w, sc.h)), np.float32(orc.beta_for_frame(sc.w, sc.h))
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    got = emdq.feature_uncertainty(f(s), f(d), f(q8), f(c), alpha, beta, f(s2)).cpu().numpy()
    want = orc.feature_uncertainty(_f32(s), _f32(d), _f32(q8), _f32(c), float(alpha), float(beta), _f32(s2))
    inl = c > 0
    # inliers: the squared error r^2 of residuals of a few px, whose FP32 field is within
    # ~3e-4 px (the FP32 field tolerance), so within 2 |r| 3e-4 ~ 1e-2 px^2; outliers: relative
    np.testing.assert_allclose(got[inl], want[inl], atol=1e-2, rtol=1e-4)
    fin = ~inl & (want < 1e30)
    np.testing.assert_allclose(got[fin], want[fin], rtol=1e-4)
