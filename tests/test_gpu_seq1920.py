"""GPU parity at the full size of the 500-frame 1920x1080 sequence (N = 5000 matches per
frame, 8192^2 canvas), in the launch configuration the sequence benchmark times: the fits
of 8 frames in one emdq_fit_batch launch and their fields and warps in one emdq_mosaic_batch
call, checked against the split calls (the BF16 fields of 4 frames in one emdq_field_batch
call, their warps in one mosaic_warp_batch call).  The oracle runs the whole fit of four of
the frames; fields are compared on sampled pixels, the canvas everywhere."""
import numpy as np
import pytest
import torch

from synth import canvas_origin, footprint_window, gt_forward, make_matches, render_frame, workload

pytestmark = pytest.mark.gpu

FRAMES = (1, 100, 200, 250, 300, 400, 450, 499)     # out to the turn, back, past the revisit
CHECKED = (1, 200, 400, 499)
BF16_TOL = 0.05                                     # px, the BF16 field tolerance of the field tests


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


@pytest.fixture(scope='module')
def seq(orc):
    sc, cfg = workload('seq1920', seed=0)
    cw, chh = cfg['canvas']
    mt = {t: make_matches(sc, t, cfg['n'], cfg['outliers'], cfg['noise']) for t in FRAMES}
    f64 = lambda a: np.float32(a).astype(np.float64)
    want = {t: orc.fit(f64(mt[t][0]), f64(mt[t][1]), sc.w, sc.h) for t in CHECKED}
    return dict(sc=sc, cfg=cfg, cw=cw, chh=chh, origin=canvas_origin(cw, chh, sc.w, sc.h),
                matches=mt, want=want, grids={t: footprint_window(sc, t, cw, chh) for t in CHECKED})


def _apply(q8, x):
    a, b, u, v, s = (q8[:, k] for k in range(5))
    n2 = a * a + b * b
    X = ((a * a - b * b) * x[:, 0] - 2 * a * b * x[:, 1] + 2 * (a * u - b * v)) / n2
    Y = (2 * a * b * x[:, 0] + (a * a - b * b) * x[:, 1] + 2 * (b * u + a * v)) / n2
    return s[:, None] * np.stack([X, Y], 1)


def test_fit_batch_of_8_at_n5000(emdq, seq):
    sc = seq['sc']
    probs = [(torch.from_numpy(seq['matches'][t][0]).cuda(), torch.from_numpy(seq['matches'][t][1]).cuda(),
              sc.w, sc.h) for t in FRAMES]
    res = emdq.emdq_fit_batch(probs)
    torch.cuda.synchronize()
    f64 = lambda a: np.float32(a).astype(np.float64)
    for t, r in zip(FRAMES, res):
        info = emdq.read_fit_info(r['info'])
        assert info['status_name'] == 'OK', (t, info)
        if t not in CHECKED:
            continue
        want = seq['want'][t]
        close = np.any(np.abs(want['dp_trace'] - 1e-3) < 2e-4)
        assert info['iters'] == want['iters'] or (close and abs(info['iters'] - want['iters']) <= 1)
        p = r['p'].cpu().numpy()
        assert np.abs(p - want['p']).max() <= 2e-3, t
        sure = np.abs(want['p'] - 0.5) > 0.1
        c = r['c'].cpu().numpy()
        np.testing.assert_array_equal((c > 0)[sure], (want['c'] > 0)[sure])
        s = f64(seq['matches'][t][0])
        dpos = np.abs(_apply(r['q'].cpu().numpy().astype(np.float64), s) -
                      _apply(want['q8'], s))[want['c'] > 0].max()
        print(f't={t}: iters {info["iters"]}, inlier row diff {dpos:.2e} px')
        assert dpos <= 2e-3


def test_field_batch_of_4_at_n5000_sampled(emdq, orc, seq):
    """The oracle's fits of the four frames (as FP32) through one emdq_field_batch call;
    4096 sampled pixels of each 2-Mpix window against the oracle's field."""
    sc = seq['sc']
    alpha = emdq.alpha_for_frame(sc.w, sc.h)
    probs = []
    for t in CHECKED:
        w = seq['want'][t]
        probs.append((torch.from_numpy(w['q8'].astype(np.float32)).cuda(),
                      torch.from_numpy(w['c'].astype(np.float32)).cuda(),
                      torch.from_numpy(seq['matches'][t][0]).cuda(), seq['grids'][t], alpha))
    got = emdq.emdq_field_batch(probs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    for t, g, pr in zip(CHECKED, got, probs):
        grid = seq['grids'][t]
        iy = rng.integers(0, grid[3], 4096)
        ix = rng.integers(0, grid[2], 4096)
        pts = np.stack([grid[0] + ix, grid[1] + iy], 1).astype(np.float64)
        w = seq['want'][t]
        want = orc.field_points(w['q8'].astype(np.float32).astype(np.float64),
                                w['c'].astype(np.float32).astype(np.float64),
                                np.float32(seq['matches'][t][0]).astype(np.float64), pts,
                                np.float64(np.float32(alpha)))
        d = np.abs(g.cpu().numpy()[iy, ix] - want)
        assert np.isfinite(d).all()
        err = d.max()
        print(f't={t}: window {grid[2]}x{grid[3]}, sampled max error {err:.3e} px')
        assert err <= BF16_TOL


def test_warp_batch_of_4_on_the_8192_canvas(emdq, orc, seq):
    """Four frames blended in one mosaic_warp_batch call through their ground-truth
    displacement (from the generator) against the oracle's warp of each in order, over the
    whole 8192^2 canvas."""
    sc = seq['sc']
    cw, chh, origin = seq['cw'], seq['chh'], seq['origin']
    rng = np.random.default_rng(11)
    canvas0 = np.zeros((chh, cw, 4), np.uint8)
    ox, oy = origin
    canvas0[oy:oy + sc.h, ox:ox + sc.w, :3] = rng.integers(0, 256, (sc.h, sc.w, 3))
    canvas0[oy:oy + sc.h, ox:ox + sc.w, 3] = 1
    frames, disps = [], []
    for t in CHECKED:
        x0, y0, gw, gh = seq['grids'][t]
        ys, xs = torch.meshgrid(torch.arange(gh, dtype=torch.float64, device='cuda') + y0,
                                torch.arange(gw, dtype=torch.float64, device='cuda') + x0, indexing='ij')
        p = torch.stack([xs, ys], -1)
        disps.append((gt_forward(sc, p, t) - p).to(torch.float32).contiguous())
        frames.append(render_frame(sc, t, device='cuda'))
    cv_g = torch.from_numpy(canvas0).cuda()
    emdq.mosaic_warp_batch(frames, disps, [seq['grids'][t] for t in CHECKED], cv_g, origin)
    cv_o = canvas0.copy()
    for t, fr, d in zip(CHECKED, frames, disps):
        assert orc.warp(fr.cpu().numpy(), d.cpu().numpy(), seq['grids'][t], cv_o, origin) == 0
    torch.cuda.synchronize()
    cv_g = cv_g.cpu().numpy()
    np.testing.assert_array_equal(cv_g[..., 3], cv_o[..., 3])
    assert int(cv_o[..., 3].max()) >= 4          # the reference and the frames overlap
    diff = np.abs(cv_g[..., :3].astype(int) - cv_o[..., :3].astype(int))
    # one field on both sides: the blend rule keeps the two canvases within 1 LSB however
    # many frames are blended (tests/blend_bound.py: ceil((w D + e + eta)/(w + 1)) = 1 for
    # D = 1 and a rounding-sized sample gap e, since w/(w + 1) < 1)
    assert diff.max() <= 1
    touched = cv_o[..., 3] > 1
    assert (diff[touched] > 0).mean() < 1e-3


def test_fused_group_of_8_equals_field_then_warp(emdq, seq):
    """The benchmark's group call on this sequence: the fields and warps of the 8 frames (their
    GPU fits; windows spread along the camera's path, so the union holds tiles that some frames
    do not meet) in one emdq_mosaic_batch call leave the 8192^2 canvas bit for bit as
    emdq_field_batch followed by mosaic_warp_batch, in frame order."""
    sc = seq['sc']
    cw, chh, origin = seq['cw'], seq['chh'], seq['origin']
    src = {t: torch.from_numpy(seq['matches'][t][0]).cuda() for t in FRAMES}
    dst = {t: torch.from_numpy(seq['matches'][t][1]).cuda() for t in FRAMES}
    fits = dict(zip(FRAMES, emdq.emdq_fit_batch([(src[t], dst[t], sc.w, sc.h) for t in FRAMES])))
    grids = {t: footprint_window(sc, t, cw, chh) for t in FRAMES}
    frames = {t: render_frame(sc, t, device='cuda') for t in FRAMES}
    alpha = emdq.alpha_for_frame(sc.w, sc.h)
    base = torch.zeros((chh, cw, 4), dtype=torch.uint8, device='cuda')
    ox, oy = origin
    base[oy:oy + sc.h, ox:ox + sc.w, :3] = 90
    base[oy:oy + sc.h, ox:ox + sc.w, 3] = 1
    want = base.clone()
    disps = emdq.emdq_field_batch([(fits[t]['q'], fits[t]['c'], src[t], grids[t], alpha) for t in FRAMES])
    emdq.mosaic_warp_batch([frames[t] for t in FRAMES], disps, [grids[t] for t in FRAMES], want, origin)
    got = base.clone()
    emdq.emdq_mosaic_batch([(fits[t]['q'], fits[t]['c'], src[t], grids[t], alpha, frames[t]) for t in FRAMES],
                           got, origin)
    torch.cuda.synchronize()
    assert torch.equal(got, want)
    touched = int((got[..., 3] > 1).sum())
    print(f'{touched} canvas pixels blended; union of the windows '
          f'{max(g[0] + g[2] for g in grids.values()) - min(g[0] for g in grids.values())} x '
          f'{max(g[1] + g[3] for g in grids.values()) - min(g[1] for g in grids.values())}')
    assert touched > sc.w * sc.h
