"""GPU parity: emdq_fit (C ABI) against the oracle's FP64 EM fit."""
import math

import numpy as np
import pytest
import torch

from synth import make_matches, make_scene, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _gpu_fit(emdq, src, dst, w, h, **kw):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    r = emdq.emdq_fit(t(src), t(dst), w, h, **kw)
    torch.cuda.synchronize()
    info = emdq.read_fit_info(r['info']) if hasattr(emdq, 'read_fit_info') else None
    return dict(q8=r['q'].cpu().numpy().astype(np.float64), c=r['c'].cpu().numpy().astype(np.float64),
                p=r['p'].cpu().numpy().astype(np.float64), info=info)


def _apply(q8, x):
    """Warp of each row applied to its own match position (the row's prediction)."""
    a, b, u, v, s = (q8[:, k] for k in range(5))
    n2 = a * a + b * b
    X = ((a * a - b * b) * x[:, 0] - 2 * a * b * x[:, 1] + 2 * (a * u - b * v)) / n2
    Y = (2 * a * b * x[:, 0] + (a * a - b * b) * x[:, 1] + 2 * (b * u + a * v)) / n2
    return s[:, None] * np.stack([X, Y], 1)


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


@pytest.mark.parametrize('name,iters', [('pair640', 3), ('seq1280', 3)])
def test_fit_fixed_iterations_parity(emdq, orc, name, iters):
    """tol 0 -> exactly `iters` EM iterations on both sides; compare every output."""
    sc, cfg = workload(name, seed=2)
    src, dst, inl = make_matches(sc, 1, cfg['n'], cfg['outliers'], cfg['noise'])
    want = orc.fit(_f32(src), _f32(dst), sc.w, sc.h, max_iters=iters, tol_p=0.0)
    got = _gpu_fit(emdq, src, dst, sc.w, sc.h, max_iters=iters, tol_p=0.0)
    assert got['info']['status_name'] == 'ENOCONV' and got['info']['iters'] == iters
    dp = np.abs(got['p'] - want['p']).max()
    dpos = np.abs(_apply(got['q8'], _f32(src)) - _apply(want['q8'], _f32(src))).max()
    ds = np.abs(got['q8'][:, 4] - want['q8'][:, 4]).max()
    print(f'{name}: max |dp| {dp:.2e}, max row-prediction diff {dpos:.2e} px, max |ds| {ds:.2e}, '
          f'sigma2 {got["info"]["sigma2"]:.6f} vs {want["sigma2"]:.6f}')
    # FP32 products (relative rounding ~6e-8) on coordinates up to ~2000 px, summed over
    # N terms: a few 1e-4 px on a row's prediction; the posteriors follow to ~1e-5
    assert dp <= 1e-4
    assert dpos <= 2e-3
    assert got['info']['sigma2'] == pytest.approx(want['sigma2'], rel=1e-5)
    assert got['info']['gamma'] == pytest.approx(want['gamma'], abs=1e-5)
    np.testing.assert_array_equal(got['q8'][:, 5:], np.tile([1, 0, 0], (len(src), 1)))


@pytest.mark.parametrize('name', ['pair640', 'seq1280'])
def test_fit_converged_parity(emdq, orc, name):
    sc, cfg = workload(name, seed=3)
    src, dst, inl = make_matches(sc, 1, cfg['n'], cfg['outliers'], cfg['noise'])
    want = orc.fit(_f32(src), _f32(dst), sc.w, sc.h)
    got = _gpu_fit(emdq, src, dst, sc.w, sc.h)
    assert want['status'] == 0 and got['info']['status_name'] == 'OK'
    # the iteration counts agree unless the oracle's last max|dp| sits at the threshold
    close = np.any(np.abs(want['dp_trace'] - 1e-3) < 2e-4)
    assert got['info']['iters'] == want['iters'] or (close and abs(got['info']['iters'] - want['iters']) <= 1)
    # inlier decisions agree wherever the oracle's posterior is not near 1/2
    sure = np.abs(want['p'] - 0.5) > 0.1
    np.testing.assert_array_equal((got['c'] > 0)[sure], (want['c'] > 0)[sure])
    dpos = np.abs(_apply(got['q8'], _f32(src)) - _apply(want['q8'], _f32(src)))[want['c'] > 0].max()
    print(f'{name}: iters {got["info"]["iters"]} vs {want["iters"]}, inlier row diff {dpos:.2e} px')
    assert dpos <= 2e-3


def test_fit_exact_similarity(emdq, orc):
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 639, (200, 2))
    th, s, t = math.radians(5), 1.05, np.array([12.0, -7.0])
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    y = s * (x @ R.T + t)
    got = _gpu_fit(emdq, x, y, 640, 480)
    assert got['info']['status_name'] == 'OK' and got['info']['iters'] == 1
    assert got['info']['sigma2'] == 0.25
    q = orc.dq_from_rt(th, *t)
    assert np.abs(got['q8'][:, :2] - q[:2]).max() < 1e-5
    assert np.abs(got['q8'][:, 4] - s).max() < 1e-5
    assert np.abs(_apply(got['q8'], x) - y).max() < 5e-3


def test_fit_small_n_and_warm_start(emdq, orc):
    sc = make_scene(9, 640, 480, 1)
    src, dst, _ = make_matches(sc, 1, 5, 0.0, 0.5)
    want = orc.fit(_f32(src), _f32(dst), 640, 480, max_iters=2, tol_p=0.0)
    got = _gpu_fit(emdq, src, dst, 640, 480, max_iters=2, tol_p=0.0)
    assert np.abs(got['p'] - want['p']).max() < 2e-3
    p0 = np.linspace(0.2, 1.0, 5)
    want = orc.fit(_f32(src), _f32(dst), 640, 480, max_iters=2, tol_p=0.0, p0=_f32(p0))
    got = _gpu_fit(emdq, src, dst, 640, 480, max_iters=2, tol_p=0.0,
                   p0=torch.tensor(p0, dtype=torch.float32, device='cuda'))
    assert np.abs(got['p'] - want['p']).max() < 2e-3
    assert got['info']['gamma'] == pytest.approx(want['gamma'], abs=1e-4)


def test_fit_device_errors(emdq):
    x = np.random.default_rng(0).uniform(0, 100, (50, 2))
    y = x.copy()
    y[3, 0] = np.nan
    got = _gpu_fit(emdq, x, y, 640, 480)
    assert got['info']['status_name'] == 'ENONFINITE'
    with pytest.raises(emdq.EmdqError):
        _gpu_fit(emdq, x[:2], y[:2], 640, 480)
    big = emdq.lib().emdq_fit_max_n() + 1
    with pytest.raises(emdq.EmdqError):
        _gpu_fit(emdq, np.zeros((big, 2)), np.zeros((big, 2)), 640, 480)


def test_fit_at_the_largest_n(emdq, orc):
    """A fit of exactly emdq_fit_max_n() matches (the shared-memory limit of one CTA) on a
    1920x1080 scene, two fixed EM iterations, against the oracle; one match more is refused."""
    n = emdq.lib().emdq_fit_max_n()
    sc = make_scene(12, 1920, 1080, 3, drift=1.0)
    src, dst, inl = make_matches(sc, 1, n, 0.3, 1.5)
    assert src.shape[0] == n
    want = orc.fit(_f32(src), _f32(dst), sc.w, sc.h, max_iters=2, tol_p=0.0)
    got = _gpu_fit(emdq, src, dst, sc.w, sc.h, max_iters=2, tol_p=0.0)
    assert got['info']['status_name'] == 'ENOCONV' and got['info']['iters'] == 2
    dp = np.abs(got['p'] - want['p']).max()
    dpos = np.abs(_apply(got['q8'], _f32(src)) - _apply(want['q8'], _f32(src)))[want['p'] > 0.5].max()
    print(f'n = {n}: max |dp| {dp:.2e}, max inlier row-prediction diff {dpos:.2e} px')
    assert dp <= 1e-4
    assert dpos <= 2e-3
    assert got['info']['sigma2'] == pytest.approx(want['sigma2'], rel=1e-5)
    s2, d2, _ = make_matches(sc, 1, n + 1, 0.3, 1.5)
    with pytest.raises(emdq.EmdqError):
        _gpu_fit(emdq, s2, d2, sc.w, sc.h)
