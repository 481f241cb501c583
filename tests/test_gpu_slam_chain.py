"""GPU: the deformation-node chain of Sec. III run end to end on a synthetic sequence, against
the generator's ground truth: nodes on the hexagonal lattice (Sec. III-E), tracked frame to frame
(EMDQ of frames t-1 -> t, Eq. 5 with App. A, Eq. 9) with ARAP smoothing (Eqs. 21-22), closed
against the reference at the end (EMDQ 0 -> T) and merged (Eqs. 12-15)."""
import math

import numpy as np
import pytest
import torch

from synth import gt_forward, make_pair_matches, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _positions(w, x0):
    """W(x0) for warp rows (torch, on the GPU's FP32 results, evaluated in float64 here)."""
    w = w.cpu().numpy().astype(np.float64)
    x0 = x0.cpu().numpy().astype(np.float64)
    nr = np.hypot(w[:, 0], w[:, 1])
    c, s, dx, dy = w[:, 0] / nr, w[:, 1] / nr, w[:, 2] / nr, w[:, 3] / nr
    tx, ty = 2 * (dx * c - dy * s), 2 * (dx * s + dy * c)
    ct, st = c * c - s * s, 2 * c * s
    return np.stack([w[:, 4] * (ct * x0[:, 0] - st * x0[:, 1] + tx),
                     w[:, 4] * (st * x0[:, 0] + ct * x0[:, 1] + ty)], 1)


def test_tracked_nodes_follow_the_ground_truth(emdq):
    sc, cfg = workload('seq1280', seed=5)
    T = 8
    dev = torch.device('cuda')
    x0 = emdq.hex_nodes(sc.w, sc.h, 40.0).to(dev)
    nn = x0.shape[0]
    ident = torch.zeros((nn, 8), device=dev)
    ident[:, 0] = ident[:, 4] = ident[:, 5] = 1.0
    alpha, beta = emdq.alpha_for_frame(sc.w, sc.h), emdq.beta_for_frame(sc.w, sc.h)
    w, s2 = ident.clone(), torch.zeros(nn, device=dev)
    s2_hist = []
    for t in range(1, T + 1):
        s, d, _, _ = make_pair_matches(sc, t - 1, t, cfg['n'], cfg['outliers'], cfg['noise'])
        st, dt = torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev)
        fit = emdq.emdq_fit(st, dt, sc.w, sc.h)
        w, s2 = emdq.node_track(x0, w, s2, fit['q'], fit['c'], st, alpha, beta)
        w = emdq.arap_smooth(x0, w, s2, alpha)
        s2_hist.append(s2.clone())
    # loop closing against the reference (the key frame 0: nodes at x0, identity warps)
    s, d, _, _ = make_pair_matches(sc, 0, T, cfg['n'], cfg['outliers'], cfg['noise'])
    st, dt = torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev)
    fit = emdq.emdq_fit(st, dt, sc.w, sc.h)
    w_loop, s2_loop = emdq.node_track(x0, ident, torch.zeros(nn, device=dev), fit['q'], fit['c'], st,
                                      alpha, beta)
    w_m, s2_m = emdq.node_merge(x0, w, s2, w_loop, s2_loop, ident, emdq.gamma_for_frame(sc.w, sc.h))
    torch.cuda.synchronize()
    truth = gt_forward(sc, x0.cpu().to(torch.float64), T).numpy()
    inside = ((truth[:, 0] > 40) & (truth[:, 0] < sc.w - 41) & (truth[:, 1] > 40) &
              (truth[:, 1] < sc.h - 41))
    err = lambda ww: np.hypot(*(_positions(ww, x0) - truth).T)[inside]
    e_track, e_loop, e_merge = err(w), err(w_loop), err(w_m)
    e_none = np.hypot(*(x0.cpu().numpy() - truth).T)[inside]
    print(f'{inside.sum()} nodes after {T} frames: median error tracked {np.median(e_track):.2f} px, '
          f'loop {np.median(e_loop):.2f}, merged {np.median(e_merge):.2f}, unmoved {np.median(e_none):.1f}')
    assert np.median(e_none) > 20.0
    assert np.median(e_track) < 3.0 and np.median(e_loop) < 3.0
    assert np.median(e_merge) <= max(np.median(e_track), np.median(e_loop)) + 0.05
    # the tracking uncertainty grows frame by frame (Eq. 9 adds Eq. 8 every step)
    grow = torch.stack(s2_hist)[:, torch.from_numpy(inside).to(dev)]
    assert bool((grow[1:] >= grow[:-1] - 1e-6).float().mean() > 0.99)
