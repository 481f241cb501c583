"""GPU parity: emdq_mosaic_batch (the fields and warps of a group of frames in one pass, the
canvas held on chip per tile) leaves the canvas bit for bit as emdq_field_batch followed by
mosaic_warp_batch, for every tile height, on the 1280x1024 sequence and on windows that are
ragged, offset, partly overlapping and disjoint; and against the oracle within the colour
bound of the blend rule."""
import numpy as np
import pytest
import torch

from blend_bound import carry, sample_gap
from synth import canvas_origin, footprint_window, make_matches, render_frame, render_reference, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


@pytest.fixture(scope='module')
def seq(emdq):
    sc, cfg = workload('seq1280', seed=3)
    cw, chh = cfg['canvas']
    origin = canvas_origin(cw, chh, sc.w, sc.h)
    T = (1, 2, 3, 4, 5)
    srcs, fits, frames, grids = [], [], [], []
    for t in T:
        s, d, _ = make_matches(sc, t, cfg['n'], cfg['outliers'], cfg['noise'])
        s, d = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
        srcs.append(s)
        fits.append(emdq.emdq_fit(s, d, sc.w, sc.h))
        frames.append(render_frame(sc, t).cuda())
        grids.append(footprint_window(sc, t, cw, chh))
    base = torch.zeros((chh, cw, 4), dtype=torch.uint8, device='cuda')
    emdq.mosaic_insert_reference(render_reference(sc).cuda(), base, origin)
    torch.cuda.synchronize()
    return dict(sc=sc, origin=origin, srcs=srcs, fits=fits, frames=frames, grids=grids, base=base,
                alpha=emdq.alpha_for_frame(sc.w, sc.h))


def _split(emdq, fits, srcs, grids, alpha, frames, canvas, origin):
    disps = emdq.emdq_field_batch([(f['q'], f['c'], s, g, alpha) for f, s, g in zip(fits, srcs, grids)])
    emdq.mosaic_warp_batch(frames, disps, grids, canvas, origin)
    return disps


@pytest.mark.parametrize('tile_rows', [16, 24, 32, 40])
def test_mosaic_batch_equals_field_then_warp_on_the_sequence(emdq, seq, tile_rows):
    k = 4
    want = seq['base'].clone()
    _split(emdq, seq['fits'][:k], seq['srcs'][:k], seq['grids'][:k], seq['alpha'], seq['frames'][:k],
           want, seq['origin'])
    got = seq['base'].clone()
    emdq.emdq_mosaic_batch([(f['q'], f['c'], s, g, seq['alpha'], fr) for f, s, g, fr in
                            zip(seq['fits'][:k], seq['srcs'][:k], seq['grids'][:k], seq['frames'][:k])],
                           got, seq['origin'], tile_rows=tile_rows)
    torch.cuda.synchronize()
    assert torch.equal(got, want)
    assert int((got[..., 3] != seq['base'][..., 3]).sum()) > 0.5 * seq['sc'].w * seq['sc'].h


def _rand_case(rng, n, w, h):
    from gpu_cases import random_rows
    src, q8 = random_rows(rng, n, w, h)
    c = np.where(rng.uniform(0, 1, n) < 0.8, rng.uniform(0.5, 1, n), 0.0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    return t(q8), t(c), t(src)


@pytest.mark.parametrize('ch', [1, 3])
def test_mosaic_batch_ragged_offset_and_disjoint_windows(emdq, ch):
    """Windows of different sizes and offsets (one far from the others, so the union holds
    tiles no window meets), frames of 640x480, counts 1..6."""
    rng = np.random.default_rng(60 + ch)
    fw, fh = 640, 480
    cw, chh = 1400, 1100
    origin = (300, 250)
    alpha = np.float32(emdq.alpha_for_frame(fw, fh))
    canvas0 = torch.from_numpy(rng.integers(0, 256, (chh, cw, 4), dtype=np.uint8)).cuda()
    canvas0[..., 3] = torch.from_numpy(rng.integers(0, 31, (chh, cw), dtype=np.uint8)).cuda()
    grids = [(-20, -30, 700, 530), (5, 7, 17, 9), (100, 200, 333, 129), (-250, -240, 130, 70),
             (600, 500, 300, 200), (0, 0, 640, 480)]
    shape = (fh, fw) if ch == 1 else (fh, fw, ch)
    for count in (1, 2, 6):
        probs, fits, srcs, frames = [], [], [], []
        for k in range(count):
            q, c, s = _rand_case(rng, int(rng.integers(50, 900)), fw, fh)
            fr = torch.from_numpy(rng.integers(0, 256, shape, dtype=np.uint8)).cuda()
            probs.append((q, c, s, grids[k], alpha, fr))
            fits.append(dict(q=q, c=c))
            srcs.append(s)
            frames.append(fr)
        want = canvas0.clone()
        _split(emdq, fits, srcs, grids[:count], alpha, frames, want, origin)
        for py in (16, 32, 40):
            got = canvas0.clone()
            emdq.emdq_mosaic_batch(probs, got, origin, tile_rows=py)
            torch.cuda.synchronize()
            assert torch.equal(got, want), (count, py)


def test_mosaic_batch_against_the_oracle(emdq, orc, seq):
    """Two frames of the sequence through emdq_mosaic_batch against the oracle's field (FP64
    from the same rows) and warp on 24 canvas rows: weights bit-exact outside the coverage
    band, colours within the blend rule's bound."""
    sc, origin = seq['sc'], seq['origin']
    ox, oy = origin
    a64 = float(np.float32(seq['alpha']))
    k = 2
    got = seq['base'].clone()
    emdq.emdq_mosaic_batch([(f['q'], f['c'], s, g, seq['alpha'], fr) for f, s, g, fr in
                            zip(seq['fits'][:k], seq['srcs'][:k], seq['grids'][:k], seq['frames'][:k])],
                           got, origin)
    disps = emdq.emdq_field_batch([(f['q'], f['c'], s, g, seq['alpha']) for f, s, g in
                                   zip(seq['fits'][:k], seq['srcs'][:k], seq['grids'][:k])])
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    want = seq['base'].cpu().numpy().copy()
    g0 = seq['grids'][0]
    rows = np.linspace(g0[1], g0[1] + g0[3] - 1, 24).round().astype(int)
    D = np.zeros((len(rows), got.shape[1], 3))
    out = np.zeros((len(rows), got.shape[1]), bool)
    for f, s, g, fr, dg_all in zip(seq['fits'][:k], seq['srcs'][:k], seq['grids'][:k], seq['frames'][:k], disps):
        q8 = f['q'].cpu().numpy().astype(np.float64)
        c = f['c'].cpu().numpy().astype(np.float64)
        s64 = s.cpu().numpy().astype(np.float64)
        frame = fr.cpu().numpy()
        x0, y0, gw, gh = g
        dga = dg_all.cpu().numpy()
        for r, y in enumerate(rows):
            if not (y0 <= y < y0 + gh):
                continue
            d_o = orc.field(q8, c, s64, (x0, y, gw, 1), a64)[0]
            before = want[y + oy, x0 + ox:x0 + ox + gw].copy()
            assert orc.warp(frame, d_o.astype(np.float32)[None], (x0, y, gw, 1), want, origin) == 0
            px = np.arange(x0, x0 + gw, dtype=np.float32)
            u_o = np.stack([px + d_o[:, 0].astype(np.float32), np.float32(y) + d_o[:, 1].astype(np.float32)], 1)
            u_g = np.stack([px + dga[y - y0, :, 0], np.float32(y) + dga[y - y0, :, 1]], 1)
            near = ((np.abs(u_o[:, 0]) < 0.05) | (np.abs(u_o[:, 0] - (sc.w - 1)) < 0.05) |
                    (np.abs(u_o[:, 1]) < 0.05) | (np.abs(u_o[:, 1] - (sc.h - 1)) < 0.05))
            cov = (u_o[:, 0] >= 0) & (u_o[:, 0] <= sc.w - 1) & (u_o[:, 1] >= 0) & (u_o[:, 1] <= sc.h - 1)
            sl = slice(x0 + ox, x0 + ox + gw)
            out[r, sl] |= near
            ok = cov & ~near
            e = sample_gap(frame, u_g, u_o)
            D[r, sl] = np.where(ok[:, None], carry(D[r, sl], before[:, 3], e), D[r, sl])
    G = got[[y + oy for y in rows]]
    W = want[[y + oy for y in rows]]
    keep = ~out
    np.testing.assert_array_equal(G[..., 3][keep], W[..., 3][keep])
    diff = np.abs(G[..., :3].astype(int) - W[..., :3].astype(int))
    assert (diff[keep] <= D[keep]).all()


def test_mosaic_batch_errors(emdq, seq):
    f, s, g, fr = seq['fits'][0], seq['srcs'][0], seq['grids'][0], seq['frames'][0]
    p = (f['q'], f['c'], s, g, seq['alpha'], fr)
    cv = seq['base'].clone()
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_mosaic_batch([p] * 17, cv, seq['origin'])
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_mosaic_batch([p], cv, seq['origin'], tile_rows=48)
    with pytest.raises(emdq.EmdqError):                     # window outside the canvas
        emdq.emdq_mosaic_batch([(f['q'], f['c'], s, (5000, 0, 10, 10), seq['alpha'], fr)], cv, seq['origin'])
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_mosaic_batch([(f['q'], f['c'], s, (0, 0, 0, 10), seq['alpha'], fr)], cv, seq['origin'])
