"""GPU parity: the fused emdq_mosaic (BF16 field + warp in one kernel) leaves the canvas
exactly as emdq_field(BF16) followed by mosaic_warp does, and matches the oracle's
field + warp within the BF16 field tolerance."""
import numpy as np
import pytest
import torch

from blend_bound import carry, sample_gap
from gpu_cases import fitted_case
from synth import canvas_origin, footprint_window, render_frame, render_reference, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _canvas_pair(emdq, sc, cfg, frame, q, c, src, grid, origin, alpha):
    cw, chh = cfg['canvas']
    base = torch.zeros((chh, cw, 4), dtype=torch.uint8, device='cuda')
    emdq.mosaic_insert_reference(render_reference(sc, device='cuda'), base, origin)
    fused = base.clone()
    emdq.emdq_mosaic(q, c, src, grid, alpha, frame, fused, origin)
    split = base.clone()
    disp = emdq.emdq_field(q, c, src, grid, alpha, precision=emdq.BF16)
    emdq.mosaic_warp(frame, disp, grid, split, origin)
    torch.cuda.synchronize()
    return base, fused, split, disp


@pytest.mark.parametrize('name', ['pair640', 'seq1280'])
def test_fused_equals_field_then_warp(emdq, orc, name):
    sc, cfg, src, dst, inl, r = fitted_case(orc, name, seed=4)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    q, c, s = t(r['q8']), t(r['c']), t(src)
    cw, chh = cfg['canvas']
    origin = canvas_origin(cw, chh, sc.w, sc.h)
    grid = footprint_window(sc, 1, cw, chh)
    frame = render_frame(sc, 1, device='cuda')
    alpha = emdq.alpha_for_frame(sc.w, sc.h)
    base, fused, split, disp = _canvas_pair(emdq, sc, cfg, frame, q, c, s, grid, origin, alpha)
    assert torch.equal(fused, split)
    changed = (fused[..., 3] != base[..., 3]).sum().item()
    assert changed > 0.5 * sc.w * sc.h


def test_fused_against_oracle_band_rule(emdq, orc):
    """Oracle field (FP64) + oracle warp vs the fused kernel: weights equal except where the
    oracle's sample position lies within the BF16 field tolerance of the frame border; every
    colour within the bound of the blend rule (tests/blend_bound.py) for the two fields'
    sample positions: ceil((e + eta) / (w + 1)) for a sample gap e onto weight w."""
    sc, cfg, src, dst, inl, r = fitted_case(orc, 'pair640', seed=5)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    q8, c = np.float32(r['q8']).astype(np.float64), np.float32(r['c']).astype(np.float64)
    s64 = np.float32(src).astype(np.float64)
    cw, chh = cfg['canvas']
    origin = canvas_origin(cw, chh, sc.w, sc.h)
    grid = footprint_window(sc, 1, cw, chh)
    frame = render_frame(sc, 1, device='cuda')
    alpha = emdq.alpha_for_frame(sc.w, sc.h)
    base, fused, split, disp = _canvas_pair(emdq, sc, cfg, frame, t(r['q8']), t(r['c']), t(src),
                                            grid, origin, alpha)
    d = orc.field(q8, c, s64, grid, float(np.float32(alpha)))
    want = base.cpu().numpy().copy()
    orc.warp(frame.cpu().numpy(), d.astype(np.float32), grid, want, origin)
    got = fused.cpu().numpy()
    ys, xs = np.mgrid[grid[1]:grid[1] + grid[3], grid[0]:grid[0] + grid[2]]
    ux, uy = xs + d[..., 0], ys + d[..., 1]
    band = 0.05
    near = ((np.abs(ux) < band) | (np.abs(ux - (sc.w - 1)) < band) |
            (np.abs(uy) < band) | (np.abs(uy - (sc.h - 1)) < band))
    sl = (slice(grid[1] + origin[1], grid[1] + origin[1] + grid[3]),
          slice(grid[0] + origin[0], grid[0] + origin[0] + grid[2]))
    wg, wo = got[sl][..., 3], want[sl][..., 3]
    assert np.array_equal(wg[~near], wo[~near])
    fr = frame.cpu().numpy()
    fr = fr.reshape(fr.shape[0], fr.shape[1], -1)
    u_o = np.stack([xs.astype(np.float32) + d[..., 0].astype(np.float32),
                    ys.astype(np.float32) + d[..., 1].astype(np.float32)], -1).reshape(-1, 2)
    dg = disp.cpu().numpy()
    u_g = np.stack([xs.astype(np.float32) + dg[..., 0], ys.astype(np.float32) + dg[..., 1]],
                   -1).reshape(-1, 2)
    cov = ((u_o[:, 0] >= 0) & (u_o[:, 0] <= sc.w - 1) & (u_o[:, 1] >= 0) & (u_o[:, 1] <= sc.h - 1))
    keep = cov & ~near.reshape(-1)
    nch = fr.shape[2]
    D = np.zeros((keep.size, nch))
    w_before = base.cpu().numpy()[sl][..., 3].reshape(-1)
    D[keep] = carry(D[keep], w_before[keep], sample_gap(fr, u_g[keep], u_o[keep]))
    diff = np.abs(got[sl][..., :nch].astype(int) - want[sl][..., :nch].astype(int)).reshape(-1, nch)
    assert (diff[~near.reshape(-1)] <= D[~near.reshape(-1)]).all()
    print(f'colour diff max {diff[keep].max()}, bound max {D[keep].max():.0f} LSB')
