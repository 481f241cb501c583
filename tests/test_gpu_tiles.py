"""GPU: the canvas-band split of one sequence leaves the canvas of the untiled run, bit for
bit.  The bands of a W-GPU run are taken one after the other on this GPU (they exchange
nothing after the fits, so running them in turn is the same computation): every frame's
field and warp on its window clipped to each band, frames in order, through the same
batched calls the benchmark's band mode makes."""
import pytest
import torch

import bench
from synth import canvas_origin, footprint_window, make_matches, render_frame, render_reference, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _blend(emdq, frames, fits, srcs, grids, canvas, origin, alpha, G=4):
    """Fields in groups of G (one emdq_field_batch call) and their warps (one
    mosaic_warp_batch call), frames in order; frames whose window is None are skipped."""
    todo = [k for k, g in enumerate(grids) if g is not None]
    for i in range(0, len(todo), G):
        grp = todo[i:i + G]
        ds = emdq.emdq_field_batch([(fits[k]['q'], fits[k]['c'], srcs[k], grids[k], alpha) for k in grp])
        emdq.mosaic_warp_batch([frames[k] for k in grp], ds, [grids[k] for k in grp], canvas, origin)


@pytest.mark.parametrize('bands', [2, 3])
def test_canvas_bands_equal_the_untiled_canvas(emdq, bands):
    sc, cfg = workload('seq1280', seed=2)
    cw, chh = 2048, 2048                      # the reference and 10 frames stay inside
    origin = canvas_origin(cw, chh, sc.w, sc.h)
    n_frames = 10
    frames, srcs, fits, grids = [], [], [], []
    for k in range(n_frames):
        t = 1 + 9 * k                         # drifting bumps: windows differ frame to frame
        s, d, _ = make_matches(sc, t, cfg['n'], cfg['outliers'], cfg['noise'])
        st, dt = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
        srcs.append(st)
        fits.append(emdq.emdq_fit(st, dt, sc.w, sc.h))
        frames.append(render_frame(sc, t, device='cuda'))
        grids.append(footprint_window(sc, t, cw, chh))
    alpha = emdq.alpha_for_frame(sc.w, sc.h)
    base = torch.zeros((chh, cw, 4), dtype=torch.uint8, device='cuda')
    emdq.mosaic_insert_reference(render_reference(sc, device='cuda'), base, origin)
    whole = base.clone()
    _blend(emdq, frames, fits, srcs, grids, whole, origin, alpha)
    tiled = base.clone()
    covered = 0
    for r in range(bands):
        band = bench.canvas_band(chh, bands, r)
        clips = [bench.clip_to_band(g, origin, band) for g in grids]
        covered += sum(c[3] for c in clips if c is not None)
        _blend(emdq, frames, fits, srcs, clips, tiled, origin, alpha)
    torch.cuda.synchronize()
    assert covered == sum(g[3] for g in grids)
    assert int((whole[..., 3] > 1).sum()) > 1_000_000      # the frames were blended
    assert torch.equal(tiled, whole)
