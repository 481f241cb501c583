#!/usr/bin/env python3
"""Benchmark of the EMDQ hot path: per frame, emdq_fit -> emdq_field -> mosaic_warp.

Workload (default): the 1280x1024 RGB8 synthetic laparoscopy sequence, N = 1000 matches
per frame with 30% outliers and 1.5 px noise, deformation bumps drifting 2 px/frame,
blended into a 4096x4096 RGBW canvas.  One step = one frame through all three calls.
Metric: frame pixels per second (Mpix/s) and the median frame latency.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32]
    python bench.py --impl reference ...   # the FP64 C oracle on the host cores

Multi-GPU (torchrun): every rank mosaics its own sequence (independent canvases, no
exchange), so the scaling is weak; rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = 'EMDQ field+warp Mpix/s at 1280x1024,N=1000 vs plain FP32 GPU; p50 frame ms'
UNIT = 'Mpix/s'
L2_FLUSH_BYTES = 256 << 20

# DRAM traffic per launch from an ncu capture of each kernel (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by kernel and tied to the hash of the source it was
# measured on: a changed kernel reports null until it is captured again.
NCU_TRAFFIC = {}


def _src_hash(name: str) -> str:
    p = os.path.join(ROOT, 'paper_2103_07414_gb300', 'csrc', name)
    return hashlib.sha256(open(p, 'rb').read()).hexdigest()[:16] if os.path.exists(p) else ''


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=30)
    ap.add_argument('--warmup', type=int, default=5)
    ap.add_argument('--impl', default='emdq', choices=['emdq', 'reference'])
    ap.add_argument('--precision', default='bf16', choices=['bf16', 'fp32'])
    ap.add_argument('--workload', default='seq1280')
    ap.add_argument('--seed', type=int, default=0)
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--no-e2e', action='store_true')
    return ap.parse_args()


def measured_peaks() -> dict:
    p = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d['hbm_gbs'], bf16_tflops=d['bf16_tflops'],
                    bf16_tflops_sustained=d.get('bf16_tflops_sustained', d['bf16_tflops']),
                    sm_max_mhz=d.get('sm_max_mhz', 2070.0), source='measured')
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0,
                sm_max_mhz=2070.0, source='fallback')


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    Q = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
         'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix='.csv')
            os.close(fd)
            self.proc = subprocess.Popen(
                ['nvidia-smi', f'--id={self.index}', f'--query-gpu={self.Q}', '--format=csv,noheader,nounits',
                 '-lms', '200'], stdout=open(self.path, 'w'), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(',')]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float('nan')
        sm = [num(r[1]) for r in rows]
        mx = max(num(r[2]) for r in rows)
        reasons = set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == 'active':
                    reasons.add(nm)
        loaded = [v for v in sm if not math.isnan(v)]
        return dict(sm_mhz=statistics.median(loaded) if loaded else None, sm_max_mhz=mx,
                    reasons=sorted(reasons), samples=len(rows))


def dist_env():
    ws = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    return ws, rank, local


def prepare_sequence(name: str, seed: int, n_frames: int, device):
    """Frames, matches and windows of the first n_frames frames of a workload (all on
    the device before timing starts)."""
    import numpy as np
    import torch
    from synth import canvas_origin, footprint_window, make_matches, render_frame, render_reference, workload
    sc, cfg = workload(name, seed=seed)
    cw, chh = cfg['canvas']
    origin = canvas_origin(cw, chh, sc.w, sc.h)
    frames, src, dst, grids = [], [], [], []
    for k in range(n_frames):
        t = 1 + (k % cfg['frames'])
        frames.append(render_frame(sc, t, device=device))
        s, d, _ = make_matches(sc, t, cfg['n'], cfg['outliers'], cfg['noise'])
        src.append(torch.from_numpy(s).to(device))
        dst.append(torch.from_numpy(d).to(device))
        grids.append(footprint_window(sc, t, cw, chh))
    ref = render_reference(sc, device=device)
    return sc, cfg, origin, ref, frames, src, dst, grids


def run_gpu(args, ws, rank, local):
    import numpy as np
    import torch
    import paper_2103_07414_gb300 as emdq

    torch.cuda.set_device(local)
    dev = torch.device('cuda', local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=dev)
    prec = emdq.BF16 if args.precision == 'bf16' else emdq.FP32
    n_frames = args.warmup + args.steps
    sc, cfg, origin, ref, frames, src, dst, grids = prepare_sequence(
        args.workload, args.seed + 1000 * rank, n_frames, dev)
    cw, chh = cfg['canvas']
    n = cfg['n']
    canvas = torch.zeros((chh, cw, 4), dtype=torch.uint8, device=dev)
    emdq.mosaic_insert_reference(ref, canvas, origin)
    alpha = emdq.alpha_for_frame(sc.w, sc.h)
    max_gw = max(g[2] for g in grids)
    max_gh = max(g[3] for g in grids)
    fit_out = dict(q=torch.empty((n, 8), device=dev), c=torch.empty(n, device=dev),
                   p=torch.empty(n, device=dev), info=torch.zeros(4, dtype=torch.int32, device=dev))
    fit_ws = torch.empty(emdq.fit_workspace_size(n), dtype=torch.uint8, device=dev)
    field_ws = torch.empty(emdq.field_workspace_size(n, max_gw, max_gh, prec), dtype=torch.uint8,
                           device=dev)
    disp_buf = torch.empty(max_gw * max_gh * 2, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(k, ev=None):
        g = grids[k]
        disp = disp_buf[: g[2] * g[3] * 2].view(g[3], g[2], 2)
        if ev: ev[0].record(stream)
        emdq.emdq_fit(src[k], dst[k], sc.w, sc.h, out=fit_out, workspace=fit_ws)
        if ev: ev[1].record(stream)
        emdq.emdq_field(fit_out['q'], fit_out['c'], src[k], g, alpha, precision=prec, out=disp,
                        workspace=field_ws)
        if ev: ev[2].record(stream)
        emdq.mosaic_warp(frames[k], disp, g, canvas, origin)
        if ev: ev[3].record(stream)

    for k in range(args.warmup):
        flush.zero_()
        step(k)
    torch.cuda.synchronize()
    infos = []
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        step(args.warmup + i, evs[i])
        infos.append(fit_out['info'].clone())
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    per = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])]
                    for e in evs])                       # ms: fit, field, warp
    frame_ms = per.sum(1)
    total_ms = float(frame_ms.sum())
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    iters = [emdq.read_fit_info(x) for x in infos]

    # end to end through the public API from pinned host buffers: H2D of the frame and the
    # matches, the three calls, D2H of the fit record and the inlier weights
    e2e = None
    if not args.no_e2e:
        hf = [f.cpu().pin_memory() for f in frames[: min(8, n_frames)]]
        hs = [s.cpu().pin_memory() for s in src[: len(hf)]]
        hd = [d.cpu().pin_memory() for d in dst[: len(hf)]]
        dfr = torch.empty_like(frames[0])
        ds, dd = torch.empty_like(src[0]), torch.empty_like(dst[0])
        h_info = torch.empty(4, dtype=torch.int32).pin_memory()
        h_c = torch.empty(n, dtype=torch.float32).pin_memory()
        e_ms = []
        for i in range(args.warmup + args.steps):
            k = i % len(hf)
            g = grids[k]
            disp = disp_buf[: g[2] * g[3] * 2].view(g[3], g[2], 2)
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dfr.copy_(hf[k], non_blocking=True)
            ds.copy_(hs[k], non_blocking=True)
            dd.copy_(hd[k], non_blocking=True)
            emdq.emdq_fit(ds, dd, sc.w, sc.h, out=fit_out, workspace=fit_ws)
            emdq.emdq_field(fit_out['q'], fit_out['c'], ds, g, alpha, precision=prec, out=disp,
                            workspace=field_ws)
            emdq.mosaic_warp(dfr, disp, g, canvas, origin)
            h_info.copy_(fit_out['info'], non_blocking=True)
            h_c.copy_(fit_out['c'], non_blocking=True)
            b.record(stream)
            b.synchronize()
            if i >= args.warmup:
                e_ms.append(a.elapsed_time(b))
        e_total = sum(e_ms)
        if ws > 1:
            t = torch.tensor([e_total], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e_total = float(t.item())
        e2e = dict(value=ws * args.steps * sc.w * sc.h / 1e6 / (e_total / 1e3), unit=UNIT,
                   p50_frame_ms=float(np.median(e_ms)),
                   h2d_bytes_per_step=int(frames[0].numel() + src[0].numel() * 4 + dst[0].numel() * 4),
                   d2h_bytes_per_step=int(16 + 4 * n))

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return None

    peaks = measured_peaks()
    phase_ms = per.mean(0)
    names = ['fit', 'field', 'warp']
    dom = int(np.argmax(phase_ms))
    win_px = float(np.mean([g[2] * g[3] for g in grids[args.warmup:]]))
    mean_iters = float(np.mean([x['iters'] for x in iters]))
    rounds = mean_iters + 1
    if names[dom] == 'fit':
        # FP32 operations per match pair: 34 in the M-step, 22 in the leave-one-out blend
        work = rounds * n * n * 56.0
        peak = 152 * 128 * 2 * peaks['sm_max_mhz'] * 1e6 / 1e12
        roof = dict(bound='alu', kernel='emdq_fit_kernel', achieved=work / (phase_ms[0] * 1e-3) / 1e12,
                    peak=peak, unit='TFLOP/s', peak_source='derived: 152 SM x 128 FP32 lanes x 2 x max clock')
    elif names[dom] == 'field':
        if prec == emdq.BF16:
            work = 2.0 * 6 * win_px * n
            roof = dict(bound='tensor', kernel='field_tc_kernel', achieved=work / (phase_ms[1] * 1e-3) / 1e12,
                        peak=peaks['bf16_tflops'], unit='TFLOP/s', peak_source=peaks['source'] + ' bf16 burst')
        else:
            work = win_px * n * 17.0
            peak = 152 * 128 * 2 * peaks['sm_max_mhz'] * 1e6 / 1e12
            roof = dict(bound='alu', kernel='field_direct_kernel', achieved=work / (phase_ms[1] * 1e-3) / 1e12,
                        peak=peak, unit='TFLOP/s', peak_source='derived: 152 SM x 128 FP32 lanes x 2 x max clock')
    else:
        work = win_px * (8 + 8) + sc.w * sc.h * sc.channels
        roof = dict(bound='hbm', kernel='mosaic_warp_kernel', achieved=work / (phase_ms[2] * 1e-3) / 1e9,
                    peak=peaks['hbm_gbs'], unit='GB/s', peak_source=peaks['source'] + ' copy')
    roof['frac'] = roof['achieved'] / roof['peak']
    tr = NCU_TRAFFIC.get(roof['kernel'])
    roof['traffic'] = tr['bytes'] if tr and tr['src'] == _src_hash(tr['file']) else None

    line = dict(
        metric=METRIC, value=ws * args.steps * sc.w * sc.h / 1e6 / (total_ms / 1e3), unit=UNIT,
        n_gpus=ws, steps=args.steps, warmup=args.warmup, ms_per_step=total_ms / args.steps,
        p50_frame_ms=float(np.median(frame_ms)), higher_is_better=True, scaling='weak',
        vs_baseline=None, dtype='bf16' if prec == emdq.BF16 else 'f32', data='synthetic',
        config=dict(workload=f'{args.workload}: 1280x1024 RGB8 frames, N={n} matches/frame, '
                    f'{int(cfg["outliers"] * 100)}% outliers, 4096x4096 RGBW canvas',
                    frame=[sc.w, sc.h], n_matches=n, canvas=list(cfg['canvas']),
                    precision=args.precision, parallelism=f'dp{ws} (independent sequences)',
                    l2='flushed before every step (256 MiB write outside the timed events)',
                    mean_window_px=win_px, mean_em_iters=mean_iters),
        phases_ms=dict(fit=float(phase_ms[0]), field=float(phase_ms[1]), warp=float(phase_ms[2])),
        wall_s=wall, roofline=roof, gpu_launches=4 * args.steps, clocks=clk, e2e=e2e,
        fit_status=sorted({x['status_name'] for x in iters}),
    )
    if not args.no_cpu_baseline:
        line['cpu_baseline'] = cpu_baseline(args, budget_s=12.0)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return line


def oracle_frame(orc, sc, cfg, frame_np, s, d, grid, canvas, origin, frac):
    """One frame through the oracle: the full fit, the field and warp on a centred band of
    `frac` of the window's rows.  Returns (fit seconds, band seconds, band rows)."""
    import numpy as np
    t0 = time.perf_counter()
    r = orc.fit(s.astype(np.float64), d.astype(np.float64), sc.w, sc.h)
    t1 = time.perf_counter()
    rows = max(1, int(round(grid[3] * frac)))
    y0 = grid[1] + (grid[3] - rows) // 2
    band = (grid[0], y0, grid[2], rows)
    disp = orc.field(r['q8'], r['c'], s.astype(np.float64), band, orc.alpha_for_frame(sc.w, sc.h))
    orc.warp(frame_np, disp.astype(np.float32), band, canvas, origin)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, rows


def cpu_baseline(args, budget_s=12.0):
    """The oracle as it stands on this host's cores: a bounded sample of the workload."""
    import numpy as np
    import oracle as orc
    from synth import canvas_origin, footprint_window, make_matches, render_frame, workload
    orc.build()
    sc, cfg = workload(args.workload, seed=args.seed)
    cw, chh = cfg['canvas']
    origin = canvas_origin(cw, chh, sc.w, sc.h)
    canvas = np.zeros((chh, cw, 4), np.uint8)
    per_frame, t_start, frames = [], time.perf_counter(), 0
    frac = 0.125
    while time.perf_counter() - t_start < budget_s or frames == 0:
        t = 1 + frames
        fr = render_frame(sc, t).numpy()
        s, d, _ = make_matches(sc, t, cfg['n'], cfg['outliers'], cfg['noise'])
        grid = footprint_window(sc, t, cw, chh)
        tf, tb, rows = oracle_frame(orc, sc, cfg, fr, s, d, grid, canvas, origin, frac)
        per_frame.append(tf + tb * grid[3] / rows)
        frames += 1
    sec = float(np.mean(per_frame))
    return dict(value=sc.w * sc.h / 1e6 / sec, unit=UNIT, cores=orc.max_threads(), kind='oracle',
                sample=f'{frames} frame(s): full EM fit + field and warp on the centred 1/8 of '
                       f'the window rows, extrapolated to the full window',
                ms_per_frame=sec * 1e3)


def run_reference(args, ws, rank):
    """--impl reference: the FP64 oracle on the host cores, rank 0 only."""
    if rank != 0:
        return None
    import numpy as np
    import oracle as orc
    from synth import canvas_origin, footprint_window, make_matches, render_frame, workload
    orc.build()
    sc, cfg = workload(args.workload, seed=args.seed)
    cw, chh = cfg['canvas']
    origin = canvas_origin(cw, chh, sc.w, sc.h)
    canvas = np.zeros((chh, cw, 4), np.uint8)
    total = args.warmup + args.steps
    # probe one frame to size the band so the whole run stays near two minutes
    fr = render_frame(sc, 1).numpy()
    s, d, _ = make_matches(sc, 1, cfg['n'], cfg['outliers'], cfg['noise'])
    grid = footprint_window(sc, 1, cw, chh)
    tf, tb, rows = oracle_frame(orc, sc, cfg, fr, s, d, grid, canvas, origin, 1 / 32)
    full_band = tb * grid[3] / rows
    frac = min(1.0, max(1 / 64, (120.0 / total - tf) / max(full_band, 1e-9)))
    times = []
    for k in range(total):
        t = 1 + (k % cfg['frames'])
        fr = render_frame(sc, t).numpy()
        s, d, _ = make_matches(sc, t, cfg['n'], cfg['outliers'], cfg['noise'])
        grid = footprint_window(sc, t, cw, chh)
        tf, tb, rows = oracle_frame(orc, sc, cfg, fr, s, d, grid, canvas, origin, frac)
        if k >= args.warmup:
            times.append(tf + tb * grid[3] / rows)
    sec = float(np.mean(times))
    value = sc.w * sc.h / 1e6 / sec
    return dict(impl='reference', metric=METRIC, value=value, unit=UNIT, n_gpus=ws,
                steps=args.steps, warmup=args.warmup, ms_per_step=sec * 1e3,
                p50_frame_ms=float(np.median(times)) * 1e3, higher_is_better=True, scaling='weak',
                vs_baseline=None, dtype='f64', data='synthetic',
                config=dict(workload=f'{args.workload}: 1280x1024 RGB8 frames, N={cfg["n"]} '
                            f'matches/frame, {int(cfg["outliers"] * 100)}% outliers, 4096x4096 canvas',
                            frame=[sc.w, sc.h], n_matches=cfg['n'], canvas=list(cfg['canvas'])),
                cpu_baseline=dict(value=value, unit=UNIT, cores=orc.max_threads(), kind='oracle',
                                  sample=f'per step: full EM fit + field and warp on {frac:.3f} of '
                                         f'the window rows, extrapolated to the full window'),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))


def main():
    args = parse_args()
    ws, rank, local = dist_env()
    if args.impl == 'reference':
        line = run_reference(args, ws, rank)
    else:
        line = run_gpu(args, ws, rank, local)
    if line is not None and rank == 0:
        print(json.dumps(line))


if __name__ == '__main__':
    main()
