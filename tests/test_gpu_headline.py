"""GPU parity of the benchmark's own batched path on the 1280x1024 sequence (N = 1000 matches
per frame, 30 % outliers, bumps drifting 2 px/frame, 4096^2 canvas), end to end against the
FP64 oracle: the learned warm start and the fits of the first 50 frames in one launch each (as
the benchmark fits a batch), then four of those frames through one emdq_field_batch call (BF16)
and one mosaic_warp_batch call (the benchmark's field group and warp group).  The oracle runs
its own chain on the same inputs: full EM fits from p = 1, FP64 fields from its own rows, and
its warp of each frame in order onto its own reference canvas.

Checks:
  - fits: every GPU fit converges; inlier labels agree wherever the oracle's posterior is
    farther than 0.1 from 1/2;
  - fields: the BF16 field of the oracle's own rows, and the field of the whole GPU chain,
    within 0.05 px of the oracle's field at 4096 sampled pixels of each window;
  - canvas: on 36 canvas rows spread over the windows, the weights are bit-exact except at
    pixels whose oracle sample position lies within 0.05 px of the frame's border (the
    coverage band), and every colour is within the bound the blend rule implies.

The colour bound (tests/blend_bound.py) is carried pixel by pixel through the frames in order:
one update moves two canvases that differ by at most D to at most ceil((w D + e + eta)/(w + 1))
apart, e the largest difference of the two samples, which the two fields' sample positions and
the frame's local pixel differences bound.
"""
import numpy as np
import pytest
import torch

from blend_bound import carry, sample_gap
from synth import canvas_origin, footprint_window, make_matches, render_frame, render_reference, workload

pytestmark = pytest.mark.gpu

FIT_FRAMES = tuple(range(1, 51))        # the benchmark's first fit launch
CHECKED = (1, 17, 34, 50)               # one field group and one warp group
BF16_TOL = 0.05                         # px, the BF16 field tolerance


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


@pytest.fixture(scope='module')
def chain(emdq, orc):
    sc, cfg = workload('seq1280', seed=0)
    cw, chh = cfg['canvas']
    origin = canvas_origin(cw, chh, sc.w, sc.h)
    mt = {t: make_matches(sc, t, cfg['n'], cfg['outliers'], cfg['noise']) for t in FIT_FRAMES}
    frames = {t: render_frame(sc, t).numpy() for t in CHECKED}       # rendered on the host
    ref = render_reference(sc).numpy()
    grids = {t: footprint_window(sc, t, cw, chh) for t in CHECKED}
    alpha = emdq.alpha_for_frame(sc.w, sc.h)

    # the GPU chain, in the benchmark's calls
    dev = 'cuda'
    srcs = [torch.from_numpy(mt[t][0]).to(dev) for t in FIT_FRAMES]
    dsts = [torch.from_numpy(mt[t][1]).to(dev) for t in FIT_FRAMES]
    p0 = emdq.warm_start(list(zip(srcs, dsts)), emdq.load_warmstart_params(dev))
    fits = emdq.emdq_fit_batch([(a, b, sc.w, sc.h, p) for a, b, p in zip(srcs, dsts, p0)])
    fit_of = dict(zip(FIT_FRAMES, fits))
    src_of = dict(zip(FIT_FRAMES, srcs))
    disps = emdq.emdq_field_batch([(fit_of[t]['q'], fit_of[t]['c'], src_of[t], grids[t], alpha)
                                   for t in CHECKED])
    canvas = torch.zeros((chh, cw, 4), dtype=torch.uint8, device=dev)
    emdq.mosaic_insert_reference(torch.from_numpy(ref).to(dev), canvas, origin)
    emdq.mosaic_warp_batch([torch.from_numpy(frames[t]).to(dev) for t in CHECKED], disps,
                           [grids[t] for t in CHECKED], canvas, origin)
    torch.cuda.synchronize()

    # the oracle's chain: its own fits from p = 1
    f64 = lambda a: np.float32(a).astype(np.float64)
    want = {t: orc.fit(f64(mt[t][0]), f64(mt[t][1]), sc.w, sc.h) for t in CHECKED}
    return dict(sc=sc, cfg=cfg, origin=origin, mt=mt, frames=frames, ref=ref, grids=grids,
                alpha=alpha, fits=fit_of, srcs=src_of,
                disps={t: d.cpu().numpy() for t, d in zip(CHECKED, disps)},
                canvas=canvas.cpu().numpy(), want=want)


def test_fits_of_one_launch_against_the_oracle(emdq, chain):
    for t, f in chain['fits'].items():
        assert emdq.read_fit_info(f['info'])['status_name'] == 'OK', t
    for t in CHECKED:
        w = chain['want'][t]
        sure = np.abs(w['p'] - 0.5) > 0.1
        c = chain['fits'][t]['c'].cpu().numpy()
        np.testing.assert_array_equal((c > 0)[sure], (w['c'] > 0)[sure])
        print(f't={t}: oracle iters {w["iters"]}, GPU iters '
              f'{emdq.read_fit_info(chain["fits"][t]["info"])["iters"]}, '
              f'{int((w["c"] > 0).sum())} inliers, {int((~sure).sum())} undecided')


def _samples(grid, rng, k=4096):
    iy, ix = rng.integers(0, grid[3], k), rng.integers(0, grid[2], k)
    return iy, ix, np.stack([grid[0] + ix, grid[1] + iy], 1).astype(np.float64)


def test_fields_sampled_against_the_oracle(emdq, orc, chain):
    """The oracle's fitted rows of the bumped frames through one emdq_field_batch call, and the
    GPU chain's own field, against the oracle's field from its rows."""
    sc, alpha = chain['sc'], chain['alpha']
    a64 = float(np.float32(alpha))
    t32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    probs = [(t32(chain['want'][t]['q8']), t32(chain['want'][t]['c']), chain['srcs'][t],
              chain['grids'][t], alpha) for t in CHECKED]
    from_oracle_rows = emdq.emdq_field_batch(probs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for t, g_rows in zip(CHECKED, from_oracle_rows):
        w = chain['want'][t]
        grid = chain['grids'][t]
        iy, ix, pts = _samples(grid, rng)
        q8, c = np.float32(w['q8']).astype(np.float64), np.float32(w['c']).astype(np.float64)
        s64 = np.float32(chain['mt'][t][0]).astype(np.float64)
        want = orc.field_points(q8, c, s64, pts, a64)
        e_rows = np.abs(g_rows.cpu().numpy()[iy, ix] - want).max()
        e_chain = np.abs(chain['disps'][t][iy, ix] - want).max()
        print(f't={t}: window {grid[2]}x{grid[3]}: field of the oracle rows {e_rows:.2e} px, '
              f'of the GPU chain {e_chain:.2e} px')
        assert e_rows <= BF16_TOL
        assert e_chain <= BF16_TOL


def test_canvas_rows_against_the_oracle_chain(orc, chain):
    sc, origin = chain['sc'], chain['origin']
    ox, oy = origin
    a64 = float(np.float32(chain['alpha']))
    grids = chain['grids']
    top = min(g[1] for g in grids.values())
    bottom = max(g[1] + g[3] for g in grids.values())
    rows = sorted(set(np.linspace(top, bottom - 1, 34).round().astype(int).tolist()) |
                  {grids[CHECKED[0]][1], grids[CHECKED[0]][1] + grids[CHECKED[0]][3] - 1})
    cw = chain['cfg']['canvas'][0]
    want = np.zeros_like(chain['canvas'])
    assert orc.insert_reference(chain['ref'], want, origin) == 0
    D = np.zeros((len(rows), cw, 3))                 # the carried colour bound
    out = np.zeros((len(rows), cw), bool)            # pixels left out (coverage band)
    for t in CHECKED:
        w = chain['want'][t]
        q8, c = np.float32(w['q8']).astype(np.float64), np.float32(w['c']).astype(np.float64)
        s64 = np.float32(chain['mt'][t][0]).astype(np.float64)
        x0, y0, gw, gh = grids[t]
        frame = chain['frames'][t]
        for r, y in enumerate(rows):
            if not (y0 <= y < y0 + gh):
                continue
            d_o = orc.field(q8, c, s64, (x0, y, gw, 1), a64)[0]
            before = want[y + oy, x0 + ox:x0 + ox + gw].copy()
            assert orc.warp(frame, d_o.astype(np.float32)[None], (x0, y, gw, 1), want, origin) == 0
            d_g = chain['disps'][t][y - y0]
            px = np.arange(x0, x0 + gw, dtype=np.float32)
            ux_o, uy_o = px + d_o[:, 0].astype(np.float32), np.float32(y) + d_o[:, 1].astype(np.float32)
            ux_g, uy_g = px + d_g[:, 0], np.float32(y) + d_g[:, 1]
            near = ((np.abs(ux_o) < BF16_TOL) | (np.abs(ux_o - (sc.w - 1)) < BF16_TOL) |
                    (np.abs(uy_o) < BF16_TOL) | (np.abs(uy_o - (sc.h - 1)) < BF16_TOL))
            cov = (ux_o >= 0) & (ux_o <= sc.w - 1) & (uy_o >= 0) & (uy_o <= sc.h - 1)
            sl = slice(x0 + ox, x0 + ox + gw)
            out[r, sl] |= near
            ok = cov & ~near
            e = sample_gap(frame, np.stack([ux_g, uy_g], 1), np.stack([ux_o, uy_o], 1))
            D[r, sl] = np.where(ok[:, None], carry(D[r, sl], before[:, 3], e), D[r, sl])
    got = chain['canvas'][[y + oy for y in rows]]
    ref = want[[y + oy for y in rows]]
    keep = ~out
    np.testing.assert_array_equal(got[..., 3][keep], ref[..., 3][keep])
    assert int(ref[..., 3].max()) == 1 + len(CHECKED)        # every frame reached these rows
    diff = np.abs(got[..., :3].astype(int) - ref[..., :3].astype(int))
    assert (diff[keep] <= D[keep]).all(), (diff[keep] - D[keep]).max()
    touched = keep & (ref[..., 3] > 1)
    print(f'{int(touched.sum())} blended pixels on {len(rows)} rows; {int(out.sum())} in the '
          f'coverage band; bound max {D[keep].max():.0f} LSB (> 1 LSB at '
          f'{(D[keep] > 1).mean():.2e} of channels); colour diff max {diff[keep].max()}, '
          f'> 1 LSB at {(diff[keep] > 1).mean():.2e}')
