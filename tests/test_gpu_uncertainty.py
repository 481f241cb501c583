"""GPU parity: emdq_uncertainty (Eq. 8) against the FP64 oracle: whole ragged windows,
sampled pixels of full-size windows (from the oracle's own fit of synthetic matches),
the no-inlier and overflow cases, and argument errors."""
import numpy as np
import pytest
import torch

from synth import footprint_window, make_matches, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _check(got, want):
    """FP32 map vs FP64 oracle: relative 1e-4 where the oracle is below 1e38, +inf on the
    GPU where the oracle is beyond the FP32 range; in between either."""
    got = np.asarray(got, dtype=np.float64)
    fin = want < 1e38
    assert np.isfinite(got[fin]).all()
    np.testing.assert_allclose(got[fin], want[fin], rtol=1e-4)
    assert np.isinf(got[want > 3.5e38]).all()


def _f32(a):
    return np.float32(a).astype(np.float64)


@pytest.mark.parametrize('n', [1, 7, 200])
def test_ragged_window_against_the_oracle(emdq, orc, n):
    rng = np.random.default_rng(n)
    src = rng.uniform(0, 640, (n, 2)).astype(np.float32)
    c = np.where(rng.uniform(0, 1, n) < 0.75, rng.uniform(0.5, 1, n), 0.0).astype(np.float32)
    c[0] = 1.0
    beta = emdq.beta_for_frame(640, 480)
    grid = (-37, -11, 251, 77)                # several 32 x 8 tiles and ragged edges
    got = emdq.emdq_uncertainty(torch.from_numpy(c).cuda(), torch.from_numpy(src).cuda(), grid, beta)
    want = orc.uncertainty(_f32(c), _f32(src), grid, float(np.float32(beta)))
    _check(got.cpu().numpy(), want)


@pytest.mark.parametrize('name', ['seq1280', 'seq1920'])
def test_full_size_window_sampled(emdq, orc, name):
    """The inliers of the oracle's fit of a frame of the sequence; 4096 sampled pixels of
    the whole window (at 1920x1080 frame 200 is the far end of the pan: most of the window
    is far from every inlier)."""
    sc, cfg = workload(name, seed=1)
    t = 5 if name == 'seq1280' else 200
    s, d, _ = make_matches(sc, t, cfg['n'], cfg['outliers'], cfg['noise'])
    fit = orc.fit(_f32(s), _f32(d), sc.w, sc.h)
    c = fit['c'].astype(np.float32)
    grid = footprint_window(sc, t, *cfg['canvas'])
    beta = emdq.beta_for_frame(sc.w, sc.h)
    got = emdq.emdq_uncertainty(torch.from_numpy(c).cuda(), torch.from_numpy(s).cuda(), grid, beta)
    rng = np.random.default_rng(3)
    iy, ix = rng.integers(0, grid[3], 4096), rng.integers(0, grid[2], 4096)
    pts = np.stack([grid[0] + ix, grid[1] + iy], 1).astype(np.float64)
    want = orc.uncertainty_points(_f32(c), _f32(s), pts, float(np.float32(beta)))
    _check(got.cpu().numpy()[iy, ix], want)
    if name == 'seq1920':
        assert (want > 3.5e38).any() and (want < 10).any()      # both regimes present


def test_no_inlier_and_empty_inputs(emdq):
    src = torch.rand((50, 2), device='cuda') * 100
    u = emdq.emdq_uncertainty(torch.zeros(50, device='cuda'), src, (0, 0, 40, 9), 1e-3)
    assert torch.isinf(u).all()
    u = emdq.emdq_uncertainty(torch.zeros(0, device='cuda'), torch.zeros((0, 2), device='cuda'),
                              (0, 0, 33, 3), 1e-3)
    assert torch.isinf(u).all()
    # an inlier on a pixel: exactly 1 there
    c = torch.zeros(50, device='cuda')
    c[7] = 0.9
    src[7] = torch.tensor([12.0, 5.0], device='cuda')
    u = emdq.emdq_uncertainty(c, src, (0, 0, 40, 9), 1e-3)
    assert u[5, 12].item() == 1.0 and (u >= 1.0).all()


def test_argument_errors(emdq):
    c = torch.ones(4, device='cuda')
    s = torch.zeros((4, 2), device='cuda')
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_uncertainty(c, s, (0, 0, 8, 8), 0.0)
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_uncertainty(c, s, (0, 0, 8, 8), float('nan'))
