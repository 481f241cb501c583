"""Rank body of the world-size-2 CPU test of the multi-rank benchmark path (gloo).

Each rank does what a GPU rank of bench.py does around its kernels: derives its own
sequence seed, builds its first frame's matches, takes the barrier and the maximum of the
timed region over ranks, and (rank 0) computes the whole-job throughput.  The fit of its
first frame runs through the FP64 oracle here (no GPU), to show that each rank's problem
is complete on its own: nothing is exchanged but the timing.
"""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def worker(rank: int, ws: int, port: int, outdir: str, fake_ms: list[float]):
    import numpy as np
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    from synth import make_matches, workload

    dist.init_process_group('gloo', init_method=f'tcp://127.0.0.1:{port}', rank=rank,
                            world_size=ws)
    seed = bench.rank_seed(0, rank)
    sc, cfg = workload('pair640', seed=seed)
    s, d, inl = make_matches(sc, 1, cfg['n'], cfg['outliers'], cfg['noise'])
    fit = oracle.fit(np.float32(s).astype(np.float64), np.float32(d).astype(np.float64), sc.w, sc.h)
    labels = fit['c'] > 0
    # each rank's first match, gathered only to check that the problems differ
    mine = torch.tensor(np.concatenate([s[0], d[0]]), dtype=torch.float64)
    got = [torch.zeros(4, dtype=torch.float64) for _ in range(ws)]
    dist.all_gather(got, mine)
    dist.barrier()
    t_max = bench.max_over_ranks(fake_ms[rank], ws, torch.device('cpu'))
    value = bench.job_mpix_per_s(ws, 100, sc.w, sc.h, t_max)
    dist.barrier()
    dist.destroy_process_group()
    out = dict(rank=rank, seed=seed, first=[g.tolist() for g in got], t_max=t_max, value=value,
               precision=float((labels & inl).sum() / max(1, labels.sum())),
               recall=float((labels & inl).sum() / inl.sum()), status=fit['status'])
    with open(os.path.join(outdir, f'rank{rank}.json'), 'w') as f:
        json.dump(out, f)


def tiled_worker(rank: int, ws: int, port: int, outdir: str, n_frames: int):
    """Rank body of the canvas-band split of one sequence: this rank fits frames k = rank mod
    W (FP64 oracle here, no GPU), the all-gather hands every rank every frame's fit rows, and
    the rank keeps the windows clipped to its band of canvas rows."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    from synth import canvas_origin, footprint_window, make_matches, workload

    dist.init_process_group('gloo', init_method=f'tcp://127.0.0.1:{port}', rank=rank,
                            world_size=ws)
    sc, cfg = workload('pair640', seed=4)
    n = cfg['n']
    cw, chh = cfg['canvas']
    origin = canvas_origin(cw, chh, sc.w, sc.h)
    local = {}
    for k in range(n_frames):
        if bench.frame_owner(k, ws) != rank:
            continue
        s, d, _ = make_matches(sc, 1 + k, n, cfg['outliers'], cfg['noise'])
        f = oracle.fit(np.float32(s).astype(np.float64), np.float32(d).astype(np.float64), sc.w, sc.h)
        local[k] = torch.from_numpy(np.concatenate([f['q8'], f['c'][:, None]], 1).astype(np.float32))
    rows = bench.gather_fit_rows(local, ws, rank, n_frames, n, torch.device('cpu'))
    band = bench.canvas_band(chh, ws, rank)
    clips = [bench.clip_to_band(footprint_window(sc, 1 + k, cw, chh), origin, band)
             for k in range(n_frames)]
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(outdir, f'rows{rank}.npy'), torch.stack(rows).numpy())
    with open(os.path.join(outdir, f'tiles{rank}.json'), 'w') as f:
        json.dump(dict(rank=rank, band=list(band), clips=[list(c) if c else None for c in clips],
                       owned=sorted(local)), f)
