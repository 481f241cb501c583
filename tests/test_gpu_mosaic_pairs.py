"""GPU parity: emdq_mosaic_pairs (the fields and warps of independent pairs fused in one pass,
each pair with its own frame size and canvas) leaves every canvas bit for bit as emdq_field
(BF16) followed by mosaic_warp of that pair: on mixed frame sizes and match counts (the
64-pair batch's recipe), at the 16-pair limit, on grayscale frames, on two calls in a row and
on pairs whose windows sit in disjoint rows of one canvas."""
import pytest
import torch

pytestmark = pytest.mark.gpu

PAD = 48


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _pairs(emdq, seed, count, channels=3):
    from synth import canvas_origin, footprint_window, mixed_pairs, render_frame, render_reference
    dev = torch.device('cuda')
    out = []
    for p in mixed_pairs(seed, count, channels=channels, n_range=(60, 3000)):
        sc = p['scene']
        cw, chh = sc.w + 2 * PAD, sc.h + 2 * PAD
        origin = canvas_origin(cw, chh, sc.w, sc.h)
        canvas = torch.zeros((chh, cw, 4), dtype=torch.uint8, device=dev)
        emdq.mosaic_insert_reference(render_reference(sc, device=dev), canvas, origin)
        src = torch.from_numpy(p['src']).to(dev)
        fit = emdq.emdq_fit(src, torch.from_numpy(p['dst']).to(dev), sc.w, sc.h)
        out.append(dict(q=fit['q'], c=fit['c'], src=src, grid=footprint_window(sc, 1, cw, chh),
                        alpha=emdq.alpha_for_frame(sc.w, sc.h), frame=render_frame(sc, 1, device=dev),
                        canvas=canvas, origin=origin))
    torch.cuda.synchronize()
    return out


def _split(emdq, x, canvas):
    disp = emdq.emdq_field(x['q'], x['c'], x['src'], x['grid'], alpha=x['alpha'], precision=emdq.BF16)
    emdq.mosaic_warp(x['frame'], disp, x['grid'], canvas, x['origin'])


def _fused(emdq, P, canvases):
    emdq.emdq_mosaic_pairs([(x['q'], x['c'], x['src'], x['grid'], x['alpha'], x['frame'], cv, x['origin'])
                            for x, cv in zip(P, canvases)])


def _check(emdq, P, rounds=1):
    want = [x['canvas'].clone() for x in P]
    got = [x['canvas'].clone() for x in P]
    for _ in range(rounds):
        for x, cv in zip(P, want):
            _split(emdq, x, cv)
        _fused(emdq, P, got)
    torch.cuda.synchronize()
    for b, (w, g) in enumerate(zip(want, got)):
        assert torch.equal(w, g), f'pair {b}: {(w != g).any(dim=2).sum().item()} canvas pixels differ'
        # the call did blend something: the frame's window changed the canvas
        assert not torch.equal(g, P[b]['canvas'])


def test_mosaic_pairs_equal_field_then_warp_on_mixed_pairs(emdq):
    P = _pairs(emdq, seed=11, count=5)
    assert len({(x['frame'].shape[1], x['frame'].shape[0]) for x in P}) >= 2   # mixed sizes
    _check(emdq, P)


def test_mosaic_pairs_at_the_limit_and_twice_in_a_row(emdq):
    P = _pairs(emdq, seed=12, count=16)
    _check(emdq, P, rounds=2)


def test_mosaic_pairs_grayscale(emdq):
    P = _pairs(emdq, seed=13, count=3, channels=1)
    _check(emdq, P)


def test_mosaic_pairs_disjoint_rows_of_one_canvas(emdq):
    """Two pairs on one canvas, the second pair's origin moved below the first one's window:
    accepted (their canvas rows do not overlap) and blended as the calls one by one."""
    P = _pairs(emdq, seed=14, count=2)
    a, b = P
    h = a['canvas'].shape[0] + b['canvas'].shape[0]
    w = max(a['canvas'].shape[1], b['canvas'].shape[1])
    big = torch.zeros((h, w, 4), dtype=torch.uint8, device='cuda')
    big[: a['canvas'].shape[0], : a['canvas'].shape[1]] = a['canvas']
    big[a['canvas'].shape[0]:, : b['canvas'].shape[1]] = b['canvas']
    b2 = dict(b, origin=(b['origin'][0], b['origin'][1] + a['canvas'].shape[0]))
    want = big.clone()
    _split(emdq, a, want)
    _split(emdq, b2, want)
    got = big.clone()
    _fused(emdq, [a, b2], [got, got])
    torch.cuda.synchronize()
    assert torch.equal(want, got)


def test_mosaic_pairs_refuses_overlapping_canvas_rows(emdq):
    P = _pairs(emdq, seed=15, count=2)
    shared = P[0]['canvas'].clone()
    with pytest.raises(emdq.EmdqError, match='EINVAL'):
        _fused(emdq, [P[0], dict(P[1], grid=P[0]['grid'], origin=P[0]['origin'])], [shared, shared])
