"""GPU parity: emdq_batch runs warm start, fits, fields and warps of a batch of pairs in
one call; every output must be bit for bit that of the same component calls made in the
documented order, and the fits must agree with the oracle."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

PAD = 64


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _mixed(emdq, seed, count, shared_canvas=False):
    from synth import canvas_origin, footprint_window, mixed_pairs, render_frame, render_reference
    dev = torch.device('cuda')
    out = []
    shared = None
    for p in mixed_pairs(seed, count, n_range=(60, 1500)):
        sc = p['scene']
        cw, chh = sc.w + 2 * PAD, sc.h + 2 * PAD
        if shared_canvas:
            cw, chh = 1920 + 2 * PAD, 1080 + 2 * PAD
        origin = canvas_origin(cw, chh, sc.w, sc.h)
        if shared_canvas and shared is not None:
            canvas = shared
        else:
            canvas = torch.zeros((chh, cw, 4), dtype=torch.uint8, device=dev)
            emdq.mosaic_insert_reference(render_reference(sc, device=dev), canvas, origin)
            shared = canvas
        out.append(dict(sc=sc, src=torch.from_numpy(p['src']).to(dev),
                        dst=torch.from_numpy(p['dst']).to(dev), frame=render_frame(sc, 1, device=dev),
                        grid=footprint_window(sc, 1, cw, chh), canvas=canvas, origin=origin))
    return out


def _components(emdq, P, warm_params, fit_ctas=None, fit_phases=None):
    """The documented order: warm start, all fits, then per group of 16 the fields and the
    warps in pair order."""
    p0 = None
    if warm_params is not None:
        p0 = emdq.warm_start([(x['src'], x['dst']) for x in P], warm_params)
    probs = [(x['src'], x['dst'], x['sc'].w, x['sc'].h) + ((p0[b],) if p0 is not None else ())
             for b, x in enumerate(P)]
    fits = emdq.emdq_fit_batch(probs, ctas=fit_ctas, phases=fit_phases)
    for g0 in range(0, len(P), 16):
        grp = list(range(g0, min(len(P), g0 + 16)))
        disps = emdq.emdq_field_batch([(fits[b]['q'], fits[b]['c'], P[b]['src'], P[b]['grid'],
                                        emdq.alpha_for_frame(P[b]['sc'].w, P[b]['sc'].h))
                                       for b in grp])
        for i, b in enumerate(grp):
            emdq.mosaic_warp(P[b]['frame'], disps[i], P[b]['grid'], P[b]['canvas'], P[b]['origin'])
    return fits


def _clone_canvases(P):
    seen = {}
    Q = []
    for x in P:
        k = x['canvas'].data_ptr()
        if k not in seen:
            seen[k] = x['canvas'].clone()
        Q.append(dict(x, canvas=seen[k]))
    return Q


@pytest.mark.parametrize('warm', [True, False])
def test_batch_equals_component_calls(emdq, warm):
    P = _mixed(emdq, 21, 20)                 # two field groups: 16 + 4
    Q = _clone_canvases(P)
    warm_params = emdq.load_warmstart_params() if warm else None
    got = emdq.emdq_batch(P, warm_params=warm_params)
    want = _components(emdq, Q, warm_params)
    torch.cuda.synchronize()
    for b in range(len(P)):
        for k in ('q', 'c', 'p', 'info'):
            assert torch.equal(got[b][k], want[b][k]), (b, k)
        # small pairs with many outliers may stop at the iteration cap
        assert emdq.read_fit_info(got[b]['info'])['status_name'] in ('OK', 'ENOCONV')
        assert torch.equal(P[b]['canvas'], Q[b]['canvas']), b


def test_batch_with_fit_phases_equals_component_calls(emdq):
    """emdq_batch_ex: the fits in phases (emdq_fit_batch_phases), the rest as emdq_batch."""
    P = _mixed(emdq, 23, 20)
    Q = _clone_canvases(P)
    warm_params = emdq.load_warmstart_params()
    got = emdq.emdq_batch(P, warm_params=warm_params, fit_phases=[5, 9, 14, 20])
    want = _components(emdq, Q, warm_params, fit_phases=[5, 9, 14, 20])
    torch.cuda.synchronize()
    for b in range(len(P)):
        for k in ('q', 'c', 'p', 'info'):
            assert torch.equal(got[b][k], want[b][k]), (b, k)
        assert torch.equal(P[b]['canvas'], Q[b]['canvas']), b


def test_pairs_sharing_a_canvas_blend_in_order(emdq):
    """Pairs that share one canvas are warped in array order (17 pairs: the order crosses
    a field-group boundary)."""
    P = _mixed(emdq, 5, 17, shared_canvas=True)
    Q = _clone_canvases(P)
    ctas = [1] * len(P)
    emdq.emdq_batch(P, fit_ctas=ctas)
    _components(emdq, Q, None, fit_ctas=ctas)
    torch.cuda.synchronize()
    assert torch.equal(P[0]['canvas'], Q[0]['canvas'])
    for b in range(len(P)):
        assert P[b]['canvas'].data_ptr() == P[0]['canvas'].data_ptr()


def test_batch_fits_match_the_oracle(emdq, orc):
    P = _mixed(emdq, 9, 6)
    got = emdq.emdq_batch(P)
    torch.cuda.synchronize()
    f64 = lambda a: a.cpu().numpy().astype(np.float64)
    for b in (0, 3, 5):
        sc = P[b]['sc']
        want = orc.fit(f64(P[b]['src']), f64(P[b]['dst']), sc.w, sc.h)
        info = emdq.read_fit_info(got[b]['info'])
        assert info['status_name'] in ('OK', 'ENOCONV') and info['iters'] == want['iters']
        assert np.abs(got[b]['p'].cpu().numpy() - want['p']).max() <= 1e-3


def test_batch_argument_errors(emdq):
    P = _mixed(emdq, 3, 2)
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_batch(P * 33)                       # 66 pairs: more than 64
    small = torch.empty(256, dtype=torch.uint8, device='cuda')
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_batch(P, workspace=small)
    bad = [dict(P[0], grid=(0, 0, 0, 16))]
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_batch(bad)
    with pytest.raises(ValueError):
        emdq.emdq_batch(P, fit_ctas=[1])
