"""GPU parity: ARAP smoothing of node warps (Sec. III-D, Eqs. 16-17, ARAP1-3, 21-22) against the
FP64 oracle on node lattices and on a few nodes moved anisotropically (where the printed,
node-centred ARAP fit and a centroid-centred fit differ), the fixed point of a common
similarity, and argument errors."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _row(orc, s, th, tx, ty):
    r = np.zeros(8)
    r[:4] = orc.dq_from_rt(th, tx, ty)
    r[4], r[5] = s, 1.0
    return r


def _pos(orc, w, x0):
    return np.array([orc.apply_warp(r[4], r[:4] / math.hypot(r[0], r[1]), x[0], x[1])
                     for r, x in zip(w, x0)])


def _f32(a):
    return np.float32(a).astype(np.float64)


@pytest.mark.parametrize('w,h,step,iters', [(640, 480, 40.0, 1), (640, 480, 40.0, 5), (1280, 1024, 30.0, 5)])
def test_arap_against_the_oracle(emdq, orc, w, h, step, iters):
    xs, ys = np.meshgrid(np.arange(0, w, step), np.arange(0, h, step))
    x0 = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.float64)
    rng = np.random.default_rng(int(step) + iters)
    wm = np.array([_row(orc, 1.03 * rng.uniform(0.99, 1.01), 0.05 + rng.normal(0, 0.01),
                        8.0 + rng.normal(0, 2), 4.0 + rng.normal(0, 2)) for _ in x0])
    s2 = rng.uniform(1, 50, len(x0))
    alpha = orc.alpha_for_frame(w, h)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    got = emdq.arap_smooth(f(x0), f(wm), f(s2), np.float32(alpha), max_iters=iters)
    torch.cuda.synchronize()
    want, costs = orc.arap_smooth(_f32(x0), _f32(wm), _f32(s2), float(np.float32(alpha)), iters)
    dpos = np.abs(_pos(orc, got.cpu().numpy().astype(np.float64), _f32(x0)) - _pos(orc, want, _f32(x0))).max()
    print(f'{len(x0)} nodes, {iters} iterations: max position difference {dpos:.2e} px')
    assert dpos <= 2e-3


@pytest.mark.parametrize('iters', [1, 3])
def test_arap_few_nodes_stretched(emdq, orc, iters):
    """Four nodes whose merged warps stretch them along x by different amounts: the ARAP warps
    are far from a common similarity, so the node-centred, weight-squared fit of the printed
    Eqs. 16-17 gives other warps than a centroid-centred one; the GPU follows the oracle."""
    x0 = np.array([[100.0, 100.0], [160.0, 100.0], [100.0, 150.0], [170.0, 170.0]])
    wm = np.array([_row(orc, 1.0, 0.0, 0.0, 0.0), _row(orc, 1.4, 0.0, -160.0 * 0.4 / 1.4, 5.0),
                   _row(orc, 1.1, 0.05, 3.0, -4.0), _row(orc, 0.9, -0.1, 25.0, 30.0)])
    s2 = np.array([10.0, 100.0, 300.0, 1.0])
    alpha = np.float32(1.0 / 80.0 ** 2)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    got = emdq.arap_smooth(f(x0), f(wm), f(s2), alpha, max_iters=iters).cpu().numpy().astype(np.float64)
    want, _ = orc.arap_smooth(_f32(x0), _f32(wm), _f32(s2), float(alpha), iters)
    dpos = np.abs(_pos(orc, got, x0) - _pos(orc, want, x0)).max()
    np.testing.assert_allclose(got[:, 4], want[:, 4], rtol=2e-6)
    assert dpos <= 1e-3, dpos


def test_common_similarity_is_kept(emdq, orc):
    xs, ys = np.meshgrid(np.arange(0, 640, 40.0), np.arange(0, 480, 40.0))
    x0 = np.stack([xs.ravel(), ys.ravel()], 1)
    S = _row(orc, 1.05, 0.08, 12.0, -7.0)
    wm = np.tile(S, (len(x0), 1))
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    got = emdq.arap_smooth(f(x0), f(wm), f(np.ones(len(x0))), np.float32(orc.alpha_for_frame(640, 480)))
    dpos = np.abs(_pos(orc, got.cpu().numpy().astype(np.float64), x0) - _pos(orc, wm, x0)).max()
    assert dpos <= 2e-3


def test_arap_argument_errors(emdq):
    z = torch.zeros((2, 2), device='cuda')
    with pytest.raises(emdq.EmdqError):
        emdq.arap_smooth(z, torch.zeros((2, 8), device='cuda'), torch.ones(2, device='cuda'), 1e-4)
    z = torch.zeros((8, 2), device='cuda')
    with pytest.raises(emdq.EmdqError):
        emdq.arap_smooth(z, torch.zeros((8, 8), device='cuda'), torch.ones(8, device='cuda'), 0.0)


def test_field_from_the_smoothed_nodes(emdq, orc):
    """Sec. III-D: once the nodes are tracked and smoothed the dense field is interpolated from
    the nodes (their warps as the rows, weight 1, reference positions as the centres) with the
    same tensor-core field; sampled pixels against the oracle's field from the same nodes."""
    xs, ys = np.meshgrid(np.arange(0, 1280, 30.0), np.arange(0, 1024, 30.0))
    x0 = np.stack([xs.ravel(), ys.ravel()], 1)
    rng = np.random.default_rng(31)
    wm = np.array([_row(orc, 1.03 * rng.uniform(0.99, 1.01), 0.05 + rng.normal(0, 0.01),
                        8.0 + rng.normal(0, 2), 4.0 + rng.normal(0, 2)) for _ in x0])
    s2 = rng.uniform(1, 50, len(x0))
    alpha = np.float32(orc.alpha_for_frame(1280, 1024))
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    wn = emdq.arap_smooth(f(x0), f(wm), f(s2), alpha)
    grid = (-20, -30, 1320, 1090)
    disp = emdq.emdq_field(wn, torch.ones(len(x0), device='cuda'), f(x0), grid, alpha, precision=emdq.BF16)
    torch.cuda.synchronize()
    iy, ix = rng.integers(0, grid[3], 4096), rng.integers(0, grid[2], 4096)
    pts = np.stack([grid[0] + ix, grid[1] + iy], 1).astype(np.float64)
    want = orc.field_points(wn.cpu().numpy().astype(np.float64), np.ones(len(x0)), _f32(x0), pts,
                            float(alpha))
    assert np.abs(disp.cpu().numpy()[iy, ix] - want).max() <= 0.05


def test_node_insertion(emdq, orc):
    """Sec. III-E: the library's lattice is the oracle's node set (breadth-first order from the
    centre), and new nodes' warps equal the oracle's weighted averages."""
    x = emdq.hex_nodes(1280, 1024, 30.0).numpy().astype(np.float64)
    want = orc.hex_nodes(1280, 1024, 30.0)
    assert len(x) == len(want)
    a = np.array(sorted(map(tuple, np.round(x, 3))))
    b = np.array(sorted(map(tuple, np.round(want, 3))))
    np.testing.assert_allclose(a, b, atol=2e-3)
    assert np.allclose(x[0], [639.5, 511.5])
    d0 = np.hypot(*(x - x[0]).T)
    assert (np.diff(d0[:7]) >= -1e-9).all() and np.allclose(d0[1:7], 30.0, atol=1e-3)
    rng = np.random.default_rng(41)
    w = np.array([_row(orc, rng.uniform(0.97, 1.03), rng.normal(0, 0.05), *rng.normal(0, 5, 2)) for _ in x])
    pts = rng.uniform(-100, 1400, (500, 2))
    alpha = np.float32(orc.alpha_for_frame(1280, 1024))
    f = lambda v: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda()
    got = emdq.node_init(f(x), f(w), f(pts), alpha).cpu().numpy().astype(np.float64)
    ref = orc.node_init(_f32(x), _f32(w), _f32(pts), float(alpha))
    dpos = np.abs(_pos(orc, got, _f32(pts)) - _pos(orc, ref, _f32(pts))).max()
    assert dpos <= 2e-3
    np.testing.assert_allclose(got[:, 4], ref[:, 4], rtol=1e-5)
