"""Training data and evaluation of the learned EM warm start (test infrastructure: the labels
and the evaluation's reference field come from the FP64 oracle).

Training data: matches of seeded 640x480 scenes (N = 200, outlier rate 10-45 %, noise
0.5-2 px); features from the library's feature kernel; labels = the FP64 oracle EMDQ's inlier
posterior at convergence (a soft label: a network that predicts the final posterior lets EM
start where it would end).  The training itself is the package's
(paper_2103_07414_gb300.training.train): the library's own forward/backward/Adam kernels
(emdq_mlp_train_step), with a cosine-decayed learning rate.

    python tests/warmstart_train.py --seeds 1000 --out warmstart_mlp.npy

writes the trained parameters (5313 float32) that the package ships as
paper_2103_07414_gb300/warmstart_mlp.npy.  `evaluate` compares plain EM with the warm-started
EM on the 1280x1024, N = 2000, 40 % outlier workload: EM iterations and field error.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def make_training_set(seeds, n=200, w=640, h=480, device='cuda'):
    """Features (GPU kernels) and labels (oracle) of len(seeds) synthetic pairs."""
    import torch

    import oracle
    import paper_2103_07414_gb300 as emdq
    from synth import make_matches, make_scene
    feats, labels = [], []
    for seed in seeds:
        g = np.random.Generator(np.random.Philox(key=[int(seed), 91]))
        out_frac = float(g.uniform(0.10, 0.45))
        noise = float(g.uniform(0.5, 2.0))
        sc = make_scene(int(seed), w, h, 1)
        s, d, _ = make_matches(sc, 1, n, out_frac, noise)
        f64 = lambda a: np.asarray(a, np.float32).astype(np.float64)
        ref = oracle.fit(f64(s), f64(d), w, h)
        st, dt = torch.from_numpy(s).to(device), torch.from_numpy(d).to(device)
        feats.append(emdq.warm_features(st, dt))
        labels.append(torch.from_numpy(ref['p'].astype(np.float32)).to(device))
    return torch.cat(feats), torch.cat(labels)


def evaluate(params, seeds=(0, 1, 2), name='warm2000', device='cuda'):
    """Plain vs warm-started EM on a workload: iterations and field RMS error vs ground truth."""
    import torch

    import oracle
    import paper_2103_07414_gb300 as emdq
    from synth import gt_forward, make_matches, workload
    rows = []
    for seed in seeds:
        sc, cfg = workload(name, seed=seed)
        s, d, inl = make_matches(sc, 1, cfg['n'], cfg['outliers'], cfg['noise'])
        st, dt = torch.from_numpy(s).to(device), torch.from_numpy(d).to(device)
        g = np.random.default_rng(seed)
        P = np.stack([g.uniform(96, sc.w - 96, 3000), g.uniform(96, sc.h - 96, 3000)], 1)
        gt = gt_forward(sc, torch.from_numpy(P), 1).numpy() - P
        alpha = float(np.float32(oracle.alpha_for_frame(sc.w, sc.h)))
        res = {}
        for mode in ('plain', 'warm'):
            p0 = emdq.warm_start_p0(st, dt, params) if mode == 'warm' else None
            r = emdq.emdq_fit(st, dt, sc.w, sc.h, p0=p0)
            info = emdq.read_fit_info(r['info'])
            q = r['q'].cpu().numpy().astype(np.float64)
            c = r['c'].cpu().numpy().astype(np.float64)
            dfield = oracle.field_points(q, c, np.float32(s).astype(np.float64), P, alpha)
            err = np.sqrt(((dfield - gt) ** 2).sum(1))
            lab = c > 0
            res[mode] = dict(iters=info['iters'], status=info['status_name'],
                             rms=float(np.sqrt((err ** 2).mean())),
                             precision=float((lab & inl).sum() / max(1, lab.sum())),
                             recall=float((lab & inl).sum() / inl.sum()))
        rows.append(res)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--seeds', type=int, default=1000)
    ap.add_argument('--steps', type=int, default=3000)
    ap.add_argument('--out', default='warmstart_mlp.npy')
    args = ap.parse_args()
    import torch
    t0 = time.time()
    feat, label = make_training_set(range(10_000, 10_000 + args.seeds))
    print(f'training set: {feat.shape[0]} matches, inlier fraction {float(label.mean()):.3f}, '
          f'{time.time() - t0:.1f} s', flush=True)
    t0 = time.time()
    from paper_2103_07414_gb300.training import train
    params, losses = train(feat, label, steps=args.steps, log_every=max(1, args.steps // 10))
    torch.cuda.synchronize()
    print(f'trained {args.steps} steps in {time.time() - t0:.2f} s; loss ' +
          ', '.join(f'{s}:{l:.4f}' for s, l in losses), flush=True)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.save(args.out, params.cpu().numpy())
    for r in evaluate(params):
        print(r, flush=True)


if __name__ == '__main__':
    main()
