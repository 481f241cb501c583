"""GPU parity: mosaic_warp (C ABI) against the oracle's warp, element by element."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    assert torch.cuda.is_available()
    return pkg


def _smooth_disp(rng, gh, gw, amp, base=(0.0, 0.0)):
    ys, xs = np.mgrid[0:gh, 0:gw].astype(np.float64)
    d = np.empty((gh, gw, 2))
    for k in range(2):
        a, b, c = rng.uniform(0.005, 0.03, 3)
        d[..., k] = base[k] + amp * np.sin(a * xs + b * ys + c * 7)
    return d.astype(np.float32)


def _compare(emdq, orc, frame, disp, grid, canvas0, origin):
    cv_o = canvas0.copy()
    assert orc.warp(frame, disp, grid, cv_o, origin) == 0
    cv_g = torch.from_numpy(canvas0).cuda()
    emdq.mosaic_warp(torch.from_numpy(frame).cuda(), torch.from_numpy(disp).cuda(), grid,
                     cv_g, origin)
    torch.cuda.synchronize()
    cv_g = cv_g.cpu().numpy()
    # coverage and weights bit-exact (u is formed in FP32 on both sides)
    np.testing.assert_array_equal(cv_g[..., 3], cv_o[..., 3])
    diff = np.abs(cv_g[..., :3].astype(int) - cv_o[..., :3].astype(int))
    assert diff.max() <= 1, diff.max()          # a rounding flip of one LSB at most
    assert (diff > 0).mean() < 1e-3
    return cv_g


@pytest.mark.parametrize('ch', [1, 3])
def test_warp_parity_ragged_window(emdq, orc, ch):
    rng = np.random.default_rng(10 + ch)
    fh, fw = 157, 211
    frame = rng.integers(0, 256, (fh, fw, ch), dtype=np.uint8)
    canvas = np.zeros((300, 400, 4), np.uint8)
    canvas[..., :3] = rng.integers(0, 256, (300, 400, 3))
    canvas[..., 3] = rng.integers(0, 31, (300, 400))
    if ch == 1:
        canvas[..., 1:3] = 0
    grid = (-13, -9, 239, 181)           # several 128-wide tiles and a ragged tail
    disp = _smooth_disp(rng, grid[3], grid[2], 6.0, base=(4.0, -3.0))
    disp[5, 7] = np.nan
    cv = _compare(emdq, orc, frame, disp, grid, canvas, (60, 50))
    assert (cv[..., 3] != canvas[..., 3]).sum() > 0.5 * fw * fh


def test_warp_zero_field_copy_and_edges(emdq, orc):
    rng = np.random.default_rng(3)
    frame = rng.integers(0, 256, (64, 130, 3), dtype=np.uint8)
    canvas = np.zeros((70, 140, 4), np.uint8)
    disp = np.zeros((64, 130, 2), np.float32)
    cv = _compare(emdq, orc, frame, disp, (0, 0, 130, 64), canvas, (5, 3))
    np.testing.assert_array_equal(cv[3:67, 5:135, :3], frame)
    # samples exactly on the last row/column are inside; just beyond are not
    disp = np.zeros((2, 3, 2), np.float32)
    disp[:, :, 0] = [[129 - 0, 0, 0], [0, 0, 0]]
    disp[0, 1, 0] = np.float32(128.001)
    _compare(emdq, orc, frame, disp, (0, 0, 3, 2), canvas, (5, 3))


def test_warp_empty_window_and_bad_window(emdq):
    frame = torch.zeros((8, 8, 3), dtype=torch.uint8, device='cuda')
    canvas = torch.zeros((16, 16, 4), dtype=torch.uint8, device='cuda')
    emdq.mosaic_warp(frame, torch.zeros((0, 5, 2), device='cuda'), (0, 0, 5, 0), canvas, (0, 0))
    with pytest.raises(emdq.EmdqError):
        emdq.mosaic_warp(frame, torch.zeros((4, 4, 2), device='cuda'), (14, 0, 4, 4), canvas, (0, 0))
    assert int(canvas.sum()) == 0


def test_insert_reference_parity(emdq, orc):
    rng = np.random.default_rng(4)
    f = rng.integers(0, 256, (33, 47, 3), dtype=np.uint8)
    cv_o = np.zeros((40, 60, 4), np.uint8)
    orc.insert_reference(f, cv_o, (6, 5))
    cv_g = torch.zeros((40, 60, 4), dtype=torch.uint8, device='cuda')
    emdq.mosaic_insert_reference(torch.from_numpy(f).cuda(), cv_g, (6, 5))
    np.testing.assert_array_equal(cv_g.cpu().numpy(), cv_o)


def test_warp_sequence_full_size_sampled(emdq, orc):
    """1280x1024 RGB into a 4096^2 canvas, the benchmark's launch: compare sampled rows."""
    from synth import workload, render_frame, footprint_window, canvas_origin
    sc, cfg = workload('seq1280', seed=0)
    frame = render_frame(sc, 7, device='cuda')
    cw, chh = cfg['canvas']
    origin = canvas_origin(cw, chh, sc.w, sc.h)
    grid = footprint_window(sc, 7, cw, chh)
    rng = np.random.default_rng(5)
    disp = _smooth_disp(rng, grid[3], grid[2], 20.0, base=(10.0, -5.0))
    canvas = torch.zeros((chh, cw, 4), dtype=torch.uint8, device='cuda')
    canvas[..., 3] = 3
    canvas[..., :3] = 100
    before = canvas.clone()
    emdq.mosaic_warp(frame, torch.from_numpy(disp).cuda(), grid, canvas, origin)
    torch.cuda.synchronize()
    fr = frame.cpu().numpy()
    rows = rng.choice(grid[3], 24, replace=False)
    for r in rows:
        y0 = grid[1] + int(r)
        sub_grid = (grid[0], y0, grid[2], 1)
        cv_o = before[y0 + origin[1]:y0 + origin[1] + 1].cpu().numpy().copy()
        orc.warp(fr, disp[r:r + 1], sub_grid, cv_o, (origin[0], -y0))
        got = canvas[y0 + origin[1]:y0 + origin[1] + 1].cpu().numpy()
        np.testing.assert_array_equal(got[..., 3], cv_o[..., 3])
        assert np.abs(got[..., :3].astype(int) - cv_o[..., :3].astype(int)).max() <= 1


@pytest.mark.parametrize('ch', [1, 3])
@pytest.mark.parametrize('count', [1, 2, 3, 5, 8])
def test_warp_batch_equals_calls_in_order(emdq, ch, count):
    """mosaic_warp_batch leaves the canvas bit for bit as count mosaic_warp calls in order:
    overlapping, disjoint, ragged and empty windows, integer and fractional shifts."""
    rng = np.random.default_rng(500 + 10 * count + ch)
    fh, fw = 97, 131
    shape = (fh, fw) if ch == 1 else (fh, fw, ch)
    canvas0 = rng.integers(0, 256, (300, 320, 4), dtype=np.uint8)
    canvas0[..., 3] = rng.integers(0, 31, (300, 320), dtype=np.uint8)
    origin = (90, 100)
    frames, disps, grids = [], [], []
    for k in range(count):
        frames.append(torch.from_numpy(rng.integers(0, 256, shape, dtype=np.uint8)).cuda())
        if k == 2:
            grid = (40, 30, 0, 10)                               # empty window
        else:
            gw, gh = int(rng.integers(20, 140)), int(rng.integers(10, 110))
            grid = (int(rng.integers(-60, 60)), int(rng.integers(-60, 60)), gw, gh)
        d = _smooth_disp(rng, grid[3], grid[2], rng.uniform(0, 6),
                         base=(float(rng.integers(-8, 8)), float(rng.uniform(-8, 8))))
        if k % 3 == 1:
            d = np.round(d)                                      # integer shifts
        disps.append(torch.from_numpy(d).cuda())
        grids.append(grid)
    cv_seq = torch.from_numpy(canvas0).cuda()
    for fr, d, g in zip(frames, disps, grids):
        emdq.mosaic_warp(fr, d, g, cv_seq, origin)
    cv_bat = torch.from_numpy(canvas0).cuda()
    emdq.mosaic_warp_batch(frames, disps, grids, cv_bat, origin)
    torch.cuda.synchronize()
    assert torch.equal(cv_seq, cv_bat)


def test_warp_batch_errors(emdq):
    fr = torch.zeros((8, 8, 3), dtype=torch.uint8, device='cuda')
    d = torch.zeros((4, 4, 2), device='cuda')
    cv = torch.zeros((32, 32, 4), dtype=torch.uint8, device='cuda')
    with pytest.raises(emdq.EmdqError):
        emdq.mosaic_warp_batch([fr] * 9, [d] * 9, [(0, 0, 4, 4)] * 9, cv, (4, 4))
    with pytest.raises(emdq.EmdqError):                    # window outside the canvas
        emdq.mosaic_warp_batch([fr], [d], [(30, 30, 4, 4)], cv, (4, 4))
    with pytest.raises(ValueError):
        emdq.mosaic_warp_batch([fr, torch.zeros((8, 9, 3), dtype=torch.uint8, device='cuda')],
                               [d, d], [(0, 0, 4, 4)] * 2, cv, (4, 4))
