#!/usr/bin/env python3
"""Benchmark of the EMDQ hot path: per frame, emdq_fit -> emdq_field -> mosaic_warp.

Workload (default): the 100-frame 1280x1024 RGB8 synthetic laparoscopy sequence, N = 1000
matches per frame with 30% outliers and 1.5 px noise, deformation bumps drifting
2 px/frame, blended into a 4096x4096 RGBW canvas.  One step = one pass over the whole
sequence, every frame through all three calls in order.  Metric: frame pixels per second
(Mpix/s) and the median frame latency.

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
NCU_TRAFFIC = {
    # emdq_field_batch on 4 frames of the 1280x1024 sequence (N = 1000, tiles of 40 pixel
    # rows): field_tc_prep_kernel 0.17-0.18 MB read + 33.1-33.9 MB written (operands written
    # back from L2) and field_tc_kernel 2.7-3.2 MB read + 44.8-46.2 MB written (the field), per
    # call; the mean of six steady-state calls over the 4 frames, per frame as the roofline's
    # unit (ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --cache-control none)
    'field': dict(bytes=20752693, file='field_tc.cu', src='59fcdfa971cfd282'),
    # emdq_mosaic_batch on the 1280x1024 sequence (calls of 13, 13, 13 and 11 frames per
    # 50-frame batch, tiles of 40 pixel rows): per 13-frame call field_tc_prep_kernel about 0.5 MB
    # read + 89 MB written (operands) and mosaic_tc_kernel about 256 MB read (operands of 13
    # frames, more than L2 holds, frames, canvas) + 68 MB written (the operands' remaining
    # write-back, the canvas); the 16 launches of the timed pass over its 100 frames, per frame
    # (ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --cache-control none)
    'mosaic': dict(bytes=32097587, file='field_tc.cu', src='8bf3f74fdf896e02'),
}


def _src_hash(name: str) -> str:
    p = os.path.join(ROOT, 'paper_2103_07414_gb300', 'csrc', name)
    return hashlib.sha256(open(p, 'rb').read()).hexdigest()[:16] if os.path.exists(p) else ''


def fused_group_size(batch: int, cap: int = 16) -> int:
    """Frames per emdq_mosaic_batch call for a fit batch of `batch` frames: the fewest calls of
    at most `cap` frames, the frames spread evenly over them (13 for 50)."""
    calls = -(-batch // cap)
    return -(-batch // calls)


def fit_phase_candidates(iters, max_iters=20):
    """Round schedules for emdq_fit_batch_phases at quantiles of `iters` (the rounds each fit
    took in a warm-up): None (one launch) first."""
    import numpy as np
    iters = np.asarray(iters, dtype=float)
    cands = [None]
    for fr in ((0.75,), (0.5, 0.8), (0.6, 0.8, 0.9), (0.5, 0.7, 0.85, 0.95)):
        ph = sorted({min(max_iters, max(1, int(np.ceil(np.quantile(iters, f))))) for f in fr} | {max_iters})
        if tuple(ph) not in cands and len(ph) > 1:
            cands.append(tuple(ph))
    return cands


def tune_fit_phases(emdq, sets, iters, max_iters=20, reps=3, margin=0.02):
    """The fit schedule of a workload: one launch or emdq_fit_batch_phases with EM round counts
    at quantiles of `iters` (the rounds its fits took in a warm-up).  sets: batches
    (problems, outs, workspace, ctas) to time on, each candidate replayed `reps` times from a
    captured CUDA graph per batch and summed over them; phases are kept only if they beat one
    launch by more than `margin`.  Returns (None or the phases, {schedule: ms per pass})."""
    import numpy as np
    import torch
    cands = fit_phase_candidates(iters, max_iters)
    st = torch.cuda.Stream()
    times = {}
    for c in cands:
        total = 0.0
        for probs, outs, ws, ctas in sets:
            kw = dict(ctas=ctas) if c is None else dict(phases=list(c))
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(st):
                emdq.emdq_fit_batch(probs, outs=outs, workspace=ws, stream=st, **kw)
                torch.cuda.synchronize()
                with torch.cuda.graph(g, stream=st):
                    for _ in range(reps):
                        emdq.emdq_fit_batch(probs, outs=outs, workspace=ws, stream=st, **kw)
            ts = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                g.replay()
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1) / reps)
            total += float(np.median(ts))
        times[c] = total
    best = min((c for c in cands if c is not None), key=times.get, default=None)
    if best is None or times[best] > (1.0 - margin) * times[None]:
        best = None
    return (None if best is None else list(best)), {
        ('one launch' if k is None else ','.join(map(str, k))): round(v, 4) for k, v in times.items()}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=20)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='emdq', choices=['emdq', 'reference'])
    ap.add_argument('--precision', default='bf16', choices=['bf16', 'fp32'])
    ap.add_argument('--workload', default='seq1280',
                    help='seq1280 (the 100-frame sequence), batch64 (64 mixed-size pairs), seq1920 '
                         '(the 500-frame 1920x1080 sequence, N=5000), or another workload of synth')
    ap.add_argument('--seed', type=int, default=0)
    ap.add_argument('--frames', type=int, default=0,
                    help='frames per step (default: the whole sequence of the workload)')
    ap.add_argument('--min-warmup-s', type=float, default=0.5,
                    help='keep warming up for at least this long (clock ramp)')
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--no-extras', action='store_true',
                    help='skip the sub-results printed beside the default seq1280 line (latency '
                         'mode, the 64-pair mixed batch, the 1920x1080 sequence)')
    ap.add_argument('--no-beside', action='store_true',
                    help='skip the calls timed beside the step (uncertainty, node tracking, ARAP)')
    ap.add_argument('--no-e2e', action='store_true')
    ap.add_argument('--no-plain', action='store_true',
                    help='skip the plain FP32 GPU comparison (per-frame emdq_fit + FP32 per-pixel '
                         'field + warp, no warm start, no batching) measured on 10 frames')
    ap.add_argument('--batch', type=int, default=0,
                    help='frames whose EM fits share one launch (1: one emdq_fit per frame; '
                         'default: the workload\'s, 50 or 8 for seq1920)')
    ap.add_argument('--no-warm', action='store_true',
                    help='plain EM (default: learned warm start when its parameters ship)')
    ap.add_argument('--fused', action='store_true',
                    help='BF16 field and warp in one emdq_mosaic call (default: emdq_field + mosaic_warp)')
    ap.add_argument('--no-graph', action='store_true',
                    help='issue every call each step (default: the pass is captured once into a '
                         'CUDA graph and replayed, removing per-call launch overhead)')
    ap.add_argument('--field-tile-rows', type=int, default=0,
                    help='tile height of the field GEMM (16, 24, 32, 40); 0: chosen by the '
                         "library's autotuner on the workload")
    ap.add_argument('--field-group', type=int, default=0,
                    help='frames per emdq_mosaic_batch (at most 16) or emdq_field_batch / '
                         'mosaic_warp_batch (at most 8; 16 for the mixed batch) call (BF16, '
                         'pipelined path); 0: for emdq_mosaic_batch the fewest calls per fit '
                         'batch, frames spread evenly (13 for batches of 50), else 4')
    ap.add_argument('--split-pairs', action='store_true',
                    help='mixed batch: each group of pairs as emdq_field_batch, then their '
                         'mosaic_warp calls on a second stream (default: one emdq_mosaic_pairs call '
                         'per group of up to 16 pairs, field and warp fused, the field never written)')
    ap.add_argument('--split-group', action='store_true',
                    help='a group of frames as emdq_field_batch, then mosaic_warp_batch on a second '
                         'stream (default for the sequence: one emdq_mosaic_batch call, field and '
                         'warp fused, the field never written)')
    ap.add_argument('--no-fit-phases', action='store_true',
                    help='every fit batch in one launch (default: the schedule, one launch or '
                         'emdq_fit_batch_phases at quantiles of the warm-up rounds, timed after '
                         'the warm-up and the fastest kept)')
    ap.add_argument('--no-pipeline', action='store_true',
                    help='field and warp of every frame on one stream (default: the warp of frame k '
                         'on a second stream, beside the field of frame k + 1)')
    ap.add_argument('--one-stream', action='store_true',
                    help='batched fields and their warps one after the other on the main stream '
                         '(default: the warps of a group on a second stream, beside the next '
                         "group's fields)")
    ap.add_argument('--hoist-warm', action='store_true',
                    help="the warm start of batch i + 1 on a third stream beside batch i's fields "
                         'and warps, as it reads only the matches (its fits still follow the blend; '
                         '+0.4 %% throughput, but a batch then starts one blend earlier, so the '
                         'frame latency grows; default: every warm start just before its fits)')
    ap.add_argument('--fit-ctas', type=int, default=0,
                    help='CTAs of one fit launch, split evenly over its frames (default: every '
                         'co-resident CTA; 152 = one per SM, which leaves room beside the GEMM '
                         'for --overlap)')
    ap.add_argument('--shard', default='sequence', choices=['sequence', 'canvas'],
                    help='N > 1: every rank its own sequence (default, weak scaling), or one '
                         'sequence split into bands of canvas rows with the fits sharded by frame '
                         'and one all-gather of the fit rows per pass (strong scaling)')
    ap.add_argument('--overlap', action='store_true',
                    help='run the next batch of fits on a second stream while the current batch is '
                         'blended (default: one stream; the cooperative fit launch occupies every '
                         'SM, so the two streams mostly serialise anyway)')
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
    """nvidia-smi sampled every 20 ms while the timed region runs."""
    Q = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
         'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self.period_ms = 20

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix='.csv')
            os.close(fd)
            self.proc = subprocess.Popen(
                ['nvidia-smi', f'--id={self.index}', f'--query-gpu={self.Q}', '--format=csv,noheader,nounits',
                 '-lms', str(self.period_ms)], stdout=open(self.path, 'w'), stderr=subprocess.DEVNULL)
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


# Multi-GPU: the path partitions by sequence.  Every rank mosaics its own independent
# sequence into its own canvas, so ranks exchange nothing on the data path; only the
# timing is combined (barrier, then the maximum over ranks of the timed region).

def rank_seed(seed: int, rank: int) -> int:
    """Seed of the sequence rank `rank` mosaics (distinct scenes and matches per rank)."""
    return seed + 1000 * rank


def max_over_ranks(x: float, ws: int, device) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mpix_per_s(ws: int, frames_per_rank: int, w: int, h: int, max_ms: float) -> float:
    """Whole-job throughput: the frame pixels all ranks processed over the slowest rank's time."""
    return ws * frames_per_rank * w * h / 1e6 / (max_ms / 1e3)


# Multi-GPU, one sequence over several GPUs (`--shard canvas`): frame k is fitted on rank
# k mod W; one all-gather per pass hands every rank every frame's fit (q rows and weights);
# rank r then computes the field and warp of every frame, in frame order, on its own band of
# canvas rows only.  A canvas pixel's updates do not depend on the window around it (the
# field at a pixel and its blend are per-pixel), so the bands assemble into the canvas an
# untiled run leaves, bit for bit.

def contiguous_runs(ks, nh: int) -> list:
    """The frames ks of a batch as runs over host rows k % nh: (first batch slot, first host
    row, count) for every stretch of consecutive host rows, so that each run is one copy."""
    out, j0 = [], 0
    for j in range(1, len(ks) + 1):
        if j == len(ks) or ks[j] % nh != ks[j - 1] % nh + 1:
            out.append((j0, ks[j0] % nh, j - j0))
            j0 = j
    return out


def canvas_band(canvas_h: int, ws: int, rank: int) -> tuple:
    """Canvas rows [y0, y1) owned by `rank` (W bands of equal height, the last takes the rest)."""
    return canvas_h * rank // ws, canvas_h * (rank + 1) // ws


def clip_to_band(grid, origin, band):
    """The rows of window `grid` (reference coordinates) that land in canvas band [y0, y1);
    None if there are none."""
    x0, y0, gw, gh = (int(v) for v in grid)
    lo = max(y0, band[0] - int(origin[1]))
    hi = min(y0 + gh, band[1] - int(origin[1]))
    return (x0, lo, gw, hi - lo) if hi > lo and gw > 0 else None


def frame_owner(k: int, ws: int) -> int:
    """The rank that fits frame k."""
    return k % ws


def gather_fit_rows(local: dict, ws: int, rank: int, n_frames: int, n: int, device):
    """Every frame's fit rows ([n, 9]: q rows and the weight c) on every rank, from the frames
    each rank fitted (`local`: frame -> [n, 9]), by one all-gather of equal-sized slabs."""
    import torch
    per = (n_frames + ws - 1) // ws
    mine = torch.zeros((per, n, 9), dtype=torch.float32, device=device)
    for j, k in enumerate(range(rank, n_frames, ws)):
        mine[j] = local[k]
    if ws == 1:
        return [mine[k] for k in range(n_frames)]
    import torch.distributed as dist
    slabs = [torch.empty_like(mine) for _ in range(ws)]
    dist.all_gather(slabs, mine)
    return [slabs[frame_owner(k, ws)][k // ws] for k in range(n_frames)]


def workload_config(args, sc, cfg, n_frames, ws) -> dict:
    """The `config` object of the JSON line (the same for both arms)."""
    cw, chh = cfg['canvas']
    return dict(workload=f'{args.workload}: {n_frames}-frame sequence of {sc.w}x{sc.h} RGB8 '
                         f'frames, N={cfg["n"]} matches/frame, {int(cfg["outliers"] * 100)}% '
                         f'outliers, {cw}x{chh} RGBW canvas; one step = one pass over the sequence',
                frame=[sc.w, sc.h], n_matches=cfg['n'], canvas=[cw, chh],
                frames_per_step=n_frames, parallelism=f'dp{ws} (independent sequences)',
                l2=f'inputs larger than L2 ({n_frames} distinct frames, '
                   f'{n_frames * sc.w * sc.h * sc.channels / 1e6:.0f} MB per step) and a '
                   f'256 MiB flush before every step, outside the timed events',
                **({'camera_pan': f'{math.hypot(*cfg["pan"]):.0f} px/frame, reversing every '
                                  f'{cfg["pan_turn"]} frames (frame {2 * cfg["pan_turn"]} revisits '
                                  f'the start)'} if cfg.get('pan_turn') else {}),
                bump_drift_px_per_frame=cfg['drift'])


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
    from synth import WORKLOADS
    n_frames = WORKLOADS[args.workload]['frames']
    if args.frames > 0:
        n_frames = min(n_frames, args.frames)
    sc, cfg, origin, ref, frames, src, dst, grids = prepare_sequence(
        args.workload, rank_seed(args.seed, rank), n_frames, dev)
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
    infos = torch.zeros((n_frames, 4), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    fused = prec == emdq.BF16 and args.fused
    B = max(1, min(args.batch or cfg.get('batch', 50), 64))
    overlap = args.overlap
    nbuf = 2 if overlap else 1            # fit outputs of two batches in flight
    c_all = torch.empty((nbuf, B, n), device=dev)       # a batch's weights in one block
    fit_outs_all = [[dict(q=torch.empty((n, 8), device=dev), c=c_all[u, b],
                          p=torch.empty(n, device=dev),
                          info=torch.zeros(4, dtype=torch.int32, device=dev))
                     for b in range(B)] for u in range(nbuf)]
    batch_ws = [torch.empty(max(256, emdq.fit_batch_workspace_size([(src[0], dst[0])] * B)),
                            dtype=torch.uint8, device=dev) for _ in range(nbuf)]
    fit_ws_all = [torch.empty(emdq.fit_workspace_size(n), dtype=torch.uint8, device=dev)
                  for _ in range(nbuf)]
    fit_stream = torch.cuda.Stream(device=dev) if overlap else stream
    warm = (not args.no_warm) and os.path.exists(emdq.WARMSTART_PARAMS)
    warm_params = emdq.load_warmstart_params(dev) if warm else None
    warm_p0 = [[torch.empty(n, device=dev) for _ in range(B)] for _ in range(nbuf)]
    hoist = warm and args.hoist_warm and not overlap
    warm_stream = torch.cuda.Stream(device=dev) if hoist else None
    warm_done = {}                  # batch -> (p0 list, event) of a warm start issued ahead

    # field / warp pipeline: the fields of a group of frames (one emdq_field_batch call on the
    # main stream) into buffer set g % 2, their warps on the warp stream after that call, in
    # frame order (the blend is order-dependent) while the next group's fields run
    piped = not fused and not args.no_pipeline
    group_fused = piped and prec == emdq.BF16 and not args.split_group
    if not (piped and prec == emdq.BF16):
        G = 1
    elif args.field_group > 0:
        G = max(1, min(16 if group_fused else 8, args.field_group))
    elif group_fused:
        G = fused_group_size(B)
    else:
        G = 4
    warp_stream = (torch.cuda.Stream(device=dev) if piped and not args.one_stream and not group_fused
                   else None)
    if piped and prec == emdq.BF16:
        zq = torch.zeros((n, 8), device=dev)
        zc = torch.zeros(n, device=dev)
        zs = torch.zeros((n, 2), device=dev)
        gws = max(emdq.field_batch_workspace_size([(zq, zc, zs, (0, 0, max_gw, max_gh), alpha)] * G),
                  emdq.mosaic_batch_workspace_size([(zq, zc, zs, (0, 0, max_gw, max_gh), alpha,
                                                     frames[0])] * G))
        grp_ws = [torch.empty(gws, dtype=torch.uint8, device=dev) for _ in range(2)]
        grp_disp = [[torch.empty(max_gw * max_gh * 2, dtype=torch.float32, device=dev)
                     for _ in range(G)] for _ in range(2)]
    elif piped:
        grp_ws = [field_ws, torch.empty_like(field_ws)]
        grp_disp = [[disp_buf], [torch.empty_like(disp_buf)]]
    slot_free = [None, None]        # warp-done event of the group that last used each set
    group_no = [0]

    def field_and_warp(fr, s_, g, fo, ev3=None):
        """One frame, not pipelined.  ev3: (field done, warp start, warp done) events."""
        if fused:
            emdq.emdq_mosaic(fo['q'], fo['c'], s_, g, alpha, fr, canvas, origin, workspace=field_ws)
            if ev3 is not None:
                for e in ev3: e.record(stream)
            return
        disp = disp_buf[: g[2] * g[3] * 2].view(g[3], g[2], 2)
        emdq.emdq_field(fo['q'], fo['c'], s_, g, alpha, precision=prec, out=disp,
                        workspace=field_ws)
        if ev3 is not None:
            ev3[0].record(stream)
            ev3[1].record(stream)
        emdq.mosaic_warp(fr, disp, g, canvas, origin)
        if ev3 is not None: ev3[2].record(stream)

    def fields_then_warps(frs, ss, gs, fos, evs3=None):
        """A group of frames, pipelined: one batched field call, then the warps."""
        two = not args.one_stream
        wst = warp_stream if two else stream      # resolved per call: capture rebinds stream
        slot = group_no[0] % 2
        group_no[0] += 1
        if group_fused:
            # one call: the group's fields and warps, the canvas words on chip per tile
            emdq.emdq_mosaic_batch([(fo['q'], fo['c'], s_, g, alpha, fr)
                                    for fo, s_, g, fr in zip(fos, ss, gs, frs)],
                                   canvas, origin, workspace=grp_ws[slot],
                                   tile_rows=args.field_tile_rows or None)
            if evs3 is not None:       # one event per call: the group's last frame blended
                evs3[-1][2].record(stream)
            return
        if two and slot_free[slot] is not None:
            stream.wait_event(slot_free[slot])
        disps = [grp_disp[slot][i][: g[2] * g[3] * 2].view(g[3], g[2], 2) for i, g in enumerate(gs)]
        if prec == emdq.BF16:
            emdq.emdq_field_batch([(fo['q'], fo['c'], s_, g, alpha) for fo, s_, g in zip(fos, ss, gs)],
                                  outs=disps, workspace=grp_ws[slot], tile_rows=args.field_tile_rows or None)
        else:
            emdq.emdq_field(fos[0]['q'], fos[0]['c'], ss[0], gs[0], alpha, precision=prec,
                            out=disps[0], workspace=grp_ws[slot])
        # dependencies through plain events (a captured graph cannot wait on the timing
        # events, which are external event nodes there)
        if evs3 is not None:
            for e3 in evs3: e3[0].record(stream)
        if two:
            fdone = torch.cuda.Event()
            fdone.record(stream)
            wst.wait_event(fdone)
        # one launch blends the group's frames in order (the first frame's events span it,
        # the others' are empty, so per-frame sums stay right)
        if evs3 is not None: evs3[0][1].record(wst)
        emdq.mosaic_warp_batch(frs, disps, gs, canvas, origin, stream=wst)
        if evs3 is not None:
            for i in range(len(frs)):
                if i: evs3[i][1].record(wst)
                evs3[i][2].record(wst)
        if two:
            wdone = torch.cuda.Event()
            wdone.record(wst)
            slot_free[slot] = wdone

    def warm_ahead(bi, ks, s_of, d_of, after, ev=None, ready=None):
        """The warm start of batch bi on the warm stream once `after` (the previous batch's
        fits, the last reader of the p0 buffers) is done; ev[0] / ev[-1] bracket it."""
        warm_stream.wait_event(after)
        if ready: ready(bi, warm_stream)
        if ev: ev[0].record(warm_stream)
        p0s = emdq.warm_start([(s_of(k), d_of(k)) for k in ks], warm_params,
                              outs=warm_p0[bi % nbuf][: len(ks)], stream=warm_stream)
        if ev: ev[-1].record(warm_stream)
        wd = torch.cuda.Event()
        wd.record(warm_stream)
        warm_done[bi] = (p0s, wd)

    fit_sched = dict(phases=None)          # set by the schedule tuner after the warm-up

    def fit_batch(bi, ks, s_of, d_of, ev=None):
        """The fits of batch bi (frames ks) on the fit stream; returns its done event.
        ev[-1] is recorded after the warm start, ev[1] before the fit launch, ev[2] after it."""
        outs = fit_outs_all[bi % nbuf]
        with torch.cuda.stream(fit_stream):
            p0s = [None] * len(ks)
            if bi in warm_done:
                p0s, wd = warm_done.pop(bi)
                fit_stream.wait_event(wd)
            elif warm:
                p0s = emdq.warm_start([(s_of(k), d_of(k)) for k in ks], warm_params,
                                      outs=warm_p0[bi % nbuf][: len(ks)], stream=fit_stream)
                if ev: ev[-1].record(fit_stream)
            if ev: ev[1].record(fit_stream)
            if B == 1:
                emdq.emdq_fit(s_of(ks[0]), d_of(ks[0]), sc.w, sc.h, p0=p0s[0], out=outs[0],
                              workspace=fit_ws_all[bi % nbuf], stream=fit_stream)
            else:
                split = None
                if args.fit_ctas > 0:
                    per, extra = divmod(args.fit_ctas, len(ks))
                    split = [max(1, per + (1 if j < extra else 0)) for j in range(len(ks))]
                emdq.emdq_fit_batch([(s_of(k), d_of(k), sc.w, sc.h, p0s[j]) for j, k in enumerate(ks)],
                                    outs=outs[: len(ks)], workspace=batch_ws[bi % nbuf],
                                    ctas=split, stream=fit_stream,
                                    phases=fit_sched['phases'] if split is None else None)
            if ev: ev[2].record(fit_stream)
            done = torch.cuda.Event()
            done.record(fit_stream)
        return done

    group_wait = [None]     # (batch, group) -> makes the main stream wait for the group's frames

    def blend_batch(bi, ks, fr_of, s_of, fit_done, ev=None):
        """Field + warp of batch bi in frame order on the main stream, after its fits."""
        stream.wait_event(fit_done)
        outs = fit_outs_all[bi % nbuf]
        if ev: ev[3].record(stream)
        if piped:
            for j0 in range(0, len(ks), G):
                if group_wait[0] is not None:
                    group_wait[0](bi, j0 // G)
                sub = list(range(j0, min(len(ks), j0 + G)))
                fields_then_warps([fr_of(ks[j]) for j in sub], [s_of(ks[j]) for j in sub],
                                  [grids[ks[j]] for j in sub], [outs[j] for j in sub],
                                  [ev[4 + 3 * j: 7 + 3 * j] for j in sub] if ev else None)
        else:
            for j, k in enumerate(ks):
                if group_wait[0] is not None:
                    group_wait[0](bi, j // G)
                field_and_warp(fr_of(k), s_of(k), grids[k], outs[j],
                               ev[4 + 3 * j: 7 + 3 * j] if ev else None)
        if warp_stream is not None:
            stream.wait_stream(warp_stream)       # the batch is blended when its warps are
            slot_free[0] = slot_free[1] = None
        for j, k in enumerate(ks):
            infos[k].copy_(outs[j]['info'])
        blended = torch.cuda.Event()
        blended.record(stream)
        return blended

    def run_batches(batches_, fr_of, s_of, d_of, evs=None, ready=None, pre_blend=None,
                    post_blend=None):
        """Fits of batch i+1 are issued before batch i is blended, so with two streams they
        overlap; a batch's fit outputs are reused two batches later, after its blend.
        ready(i, stream): makes the stream wait for batch i's matches; pre_blend(i) /
        post_blend(i): issued just before / after batch i's blend (inputs arriving from the
        host, results going back)."""
        blended = [None] * len(batches_)
        done = [None] * len(batches_)
        def blend(i, ks):
            if pre_blend: pre_blend(i)
            blended[i] = blend_batch(i, ks, fr_of, s_of, done[i], evs[i] if evs else None)
            if post_blend: post_blend(i)
        def issue_fit(i):
            if ready: ready(i, fit_stream)
            if i >= nbuf and blended[i - nbuf] is not None:
                fit_stream.wait_event(blended[i - nbuf])
            if evs is not None and i not in warm_done:
                evs[i][0].record(fit_stream)
            done[i] = fit_batch(i, batches_[i], s_of, d_of, evs[i] if evs is not None else None)
        issue_fit(0)
        for i, ks in enumerate(batches_):
            if i + 1 < len(batches_):
                if not overlap:
                    if hoist:
                        warm_ahead(i + 1, batches_[i + 1], s_of, d_of, done[i],
                                   evs[i + 1] if evs is not None else None, ready)
                    blend(i, ks)
                    issue_fit(i + 1)
                    continue
                issue_fit(i + 1)
            blend(i, ks)
        stream.wait_stream(fit_stream)

    batches = [list(range(k0, min(n_frames, k0 + B))) for k0 in range(0, n_frames, B)]

    def one_pass(evs=None):
        fit_stream.wait_stream(stream)        # after the L2 flush
        run_batches(batches, lambda k: frames[k], lambda k: src[k], lambda k: dst[k], evs)

    # warm-up: W passes, and at least half a second of work so clocks have ramped
    t0 = time.perf_counter()
    w = 0
    while w < args.warmup or time.perf_counter() - t0 < args.min_warmup_s:
        flush.zero_()
        one_pass()
        torch.cuda.synchronize()
        w += 1
    # the fit schedule: one launch per batch or emdq_fit_batch_phases at quantiles of the
    # rounds the fits took in the warm-up, each timed on whole passes of the step (the fit
    # inside the step runs slower than alone, so a fit timed alone is no guide); phases are
    # kept only if they beat one launch by more than 2 %
    fit_tune = None
    if B > 1 and args.fit_ctas == 0 and not args.no_fit_phases:
        # each candidate schedule timed on whole passes of the step (untimed pass, then two)
        times = {}
        for c in fit_phase_candidates(infos[:, 1].cpu().numpy()):
            fit_sched['phases'] = None if c is None else list(c)
            ts = []
            for r in range(3):
                flush.zero_()
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record()
                one_pass()
                b_.record()
                b_.synchronize()
                if r:
                    ts.append(a_.elapsed_time(b_))
            times[c] = float(np.mean(ts))
        best = min((c for c in times if c is not None), key=times.get, default=None)
        ph = None if best is None or times[best] > 0.98 * times[None] else list(best)
        ms = {('one launch' if k is None else ','.join(map(str, k))): round(v, 4) for k, v in times.items()}
        fit_sched['phases'] = ph
        fit_tune = dict(chosen='one launch' if ph is None else ph, ms_per_pass=ms)
    # the field tile height for this sequence's field groups, chosen by the library's
    # autotuner on the last batch's first group (recorded per size class, so the calls below,
    # and the graph captured from them, use it)
    field_tune = None
    if group_fused:
        field_tune = dict(call='emdq_mosaic_batch', tile_rows=args.field_tile_rows or 'library default')
    elif piped and prec == emdq.BF16:
        lb = len(batches) - 1
        ks_t = batches[lb][:G]
        fo_t = fit_outs_all[lb % nbuf]
        probs_t = [(fo_t[j]['q'], fo_t[j]['c'], src[k], grids[k], alpha) for j, k in enumerate(ks_t)]
        outs_t = [grp_disp[0][i][: grids[k][2] * grids[k][3] * 2].view(grids[k][3], grids[k][2], 2)
                  for i, k in enumerate(ks_t)]
        if args.field_tile_rows:
            py = args.field_tile_rows
            field_tune = dict(tile_rows=py, chosen='by --field-tile-rows')
        else:
            py, ms = emdq.field_batch_autotune(probs_t, reps=5, outs=outs_t, workspace=grp_ws[0])
            field_tune = dict(tile_rows=py, ms_per_call=ms, frames_per_call=len(ks_t))
    def new_events(external=False):
        # external: recorded as real event nodes when captured into a CUDA graph, so they
        # still time the replay
        kw = dict(external=True) if external else {}
        return [[torch.cuda.Event(enable_timing=True, **kw) for _ in range(5 + 3 * len(ks))]
                for ks in batches]

    # per batch e[0]: its fits issued and e[1]: warm start done, e[2]: fits done (all on the
    # fit stream); e[3]: its blend starts (main stream, after the fits); e[4 + 3j]: frame j's
    # field done (main stream), e[5 + 3j] / e[6 + 3j]: its warp starts / is done (warp
    # stream).  Frame latency = e[0] -> e[6 + 3j].  Kernel durations are taken on the stream
    # each kernel runs on.
    lat_ms, pass_ms = [], []
    warm_ms, fit_ms, field_ms, warp_ms = [], [], [], []
    fit_launch_frames = []

    def collect(step):
        for bi, e in enumerate(step):
            nb = (len(e) - 5) // 3
            warm_ms.append(e[0].elapsed_time(e[-1]) if warm else 0.0)
            fit_ms.append(e[1].elapsed_time(e[2]))
            fit_launch_frames.append(batches[bi])
            prev = e[3]
            if group_fused:
                # one event per group call: the call's span goes to its first frame (per-frame
                # sums stay right), every frame of the group is done when the call is
                for j0 in range(0, nb, G):
                    last = e[6 + 3 * (min(nb, j0 + G) - 1)]
                    for j in range(j0, min(nb, j0 + G)):
                        field_ms.append(prev.elapsed_time(last) if j == j0 else 0.0)
                        warp_ms.append(0.0)
                        lat_ms.append(e[0].elapsed_time(last))
                    prev = last
                continue
            for j in range(nb):
                field_ms.append(prev.elapsed_time(e[4 + 3 * j]))
                warp_ms.append(e[5 + 3 * j].elapsed_time(e[6 + 3 * j]))
                lat_ms.append(e[0].elapsed_time(e[6 + 3 * j]))
                prev = e[4 + 3 * j]

    # CUDA graph of one pass (one stream): captured once, replayed every step
    graph, graph_note, gevs = None, None, None
    if not args.no_graph:
        saved = (stream, fit_stream)
        try:
            gevs = new_events(external=True)
            cap = torch.cuda.Stream(device=dev)
            cap.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            stream = fit_stream = cap
            with torch.cuda.graph(g, stream=cap):
                run_batches(batches, lambda k: frames[k], lambda k: src[k], lambda k: dst[k], gevs)
            graph = g
        except Exception as ex:                      # capture refused: issue calls directly
            graph_note = f'capture failed, calls issued directly: {type(ex).__name__}: {ex}'[:300]
        stream, fit_stream = saved
        warm_done.clear()
        torch.cuda.synchronize()
        if graph is not None:                        # one untimed replay
            flush.zero_()
            graph.replay()
            torch.cuda.synchronize()
    evs = [new_events() for _ in range(args.steps)] if graph is None else None
    outer = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.1)
    t_wall = time.perf_counter()
    all_infos = []
    for i in range(args.steps):
        flush.zero_()
        if graph is not None:
            outer[i][0].record()
            graph.replay()
            outer[i][1].record()
            all_infos.append(infos.clone())
            # the graph's events are re-recorded by every replay: read them now (the wait
            # falls between timed steps)
            outer[i][1].synchronize()
            if gevs is not None:
                try:
                    collect(gevs)
                except RuntimeError as ex:       # no timing from inside the graph
                    gevs = None
                    graph_note = f'per-kernel times from untimed direct passes: {ex}'[:200]
            pass_ms.append(outer[i][0].elapsed_time(outer[i][1]))
        else:
            one_pass(evs[i])
            all_infos.append(infos.clone())
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    if graph is None:
        # step time: first fit issue -> last warp of the pass
        for step in evs:
            collect(step)
            pass_ms.append(step[0][0].elapsed_time(step[-1][-2]))
    elif gevs is None:
        # the graph's events could not be read: time the kernels on direct passes instead
        for step in [new_events() for _ in range(min(3, args.steps))]:
            flush.zero_()
            one_pass(step)
            torch.cuda.synchronize()
            collect(step)
    total_ms = float(np.sum(pass_ms))
    frame_ms = np.array(lat_ms)
    total_ms = max_over_ranks(total_ms, ws, dev)
    iv = torch.stack(all_infos).view(-1, 4).cpu()
    iters = iv[:, 1].numpy()
    statuses = sorted({emdq.STATUS.get(int(v), '?') for v in iv[:, 0].tolist()})
    total_frames = args.steps * n_frames

    # the uncertainty map of Eq. 8 (not part of the step): emdq_uncertainty on every frame's
    # window from the fits of the first batch, timed alone on the main stream
    unc = None
    if rank == 0 and not args.no_beside:
        fit_batch(0, batches[0], lambda k: src[k], lambda k: dst[k])
        torch.cuda.synchronize()
        outs0 = fit_outs_all[0]
        beta = emdq.beta_for_frame(sc.w, sc.h)
        umap = torch.empty(max_gw * max_gh, dtype=torch.float32, device=dev)
        ks0 = batches[0]

        def unc_pass():
            for j, k in enumerate(ks0):
                g = grids[k]
                emdq.emdq_uncertainty(outs0[j]['c'], src[k], g, beta, out=umap[: g[2] * g[3]].view(g[3], g[2]))

        unc_pass()
        u_ms = []
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            unc_pass()
            b.record(stream)
            b.synchronize()
            u_ms.append(a.elapsed_time(b) / len(ks0))
        upx = float(np.mean([grids[k][2] * grids[k][3] for k in ks0]))
        unc = dict(call='emdq_uncertainty (Eq. 8), one call per frame, not part of the step',
                   ms_per_frame=float(np.median(u_ms)), window_mpix_per_s=upx / 1e3 / float(np.median(u_ms)),
                   bound='latency', frames=len(ks0))
        # node tracking (Eq. 5, App. A, Eq. 9) of a 30-px node lattice over the frame
        xs, ys = np.meshgrid(np.arange(0, sc.w, 30.0), np.arange(0, sc.h, 30.0))
        x0n = torch.tensor(np.stack([xs.ravel(), ys.ravel()], 1), dtype=torch.float32, device=dev)
        nn = x0n.shape[0]
        wn = torch.zeros((nn, 8), device=dev)
        wn[:, 0] = 1.0
        wn[:, 4] = 1.0
        wn[:, 5] = 1.0
        s2n = torch.ones(nn, device=dev)
        alpha_n = emdq.alpha_for_frame(sc.w, sc.h)

        def node_pass():
            w_, v_ = wn, s2n
            for j, k in enumerate(ks0):
                w_, v_ = emdq.node_track(x0n, w_, v_, outs0[j]['q'], outs0[j]['c'], src[k], alpha_n, beta)
            return w_, v_

        node_pass()
        n_ms = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            node_pass()
            b.record(stream)
            b.synchronize()
            n_ms.append(a.elapsed_time(b) / len(ks0))
        unc['node_track'] = dict(call='emdq_node_track (Eq. 5, App. A, Eq. 9), one call per frame',
                                 nodes=nn, ms_per_frame=float(np.median(n_ms)))
        # ARAP smoothing (Sec. III-D, 5 iterations) of the tracked lattice
        w_t, s2_t = node_pass()
        arap_ws = torch.empty(emdq.lib().emdq_arap_workspace_size(nn), dtype=torch.uint8, device=dev)
        emdq.arap_smooth(x0n, w_t, s2_t, alpha_n, 5, workspace=arap_ws)
        a_ms = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            emdq.arap_smooth(x0n, w_t, s2_t, alpha_n, 5, workspace=arap_ws)
            b.record(stream)
            b.synchronize()
            a_ms.append(a.elapsed_time(b))
        unc['arap_smooth'] = dict(call='emdq_arap_smooth (Eqs. 16-17, ARAP1-3, 21-22), 5 iterations', nodes=nn,
                                  ms_per_call=float(np.median(a_ms)))

    # end to end through the public API from pinned host buffers: every frame and its
    # matches in pinned host memory; per batch one H2D copy of each match array and one of
    # the frames of each field group (split where the host rows wrap) on a copy stream, into
    # two device slots used alternately, so a batch's copies run beside the previous batch's
    # compute; a batch's fits wait for its matches only, each group's fused call for that
    # group's frames; after its blend the D2H of its fit records and weights, and the copies
    # of the batch two ahead into the freed slot
    e2e = None
    if not args.no_e2e:
        nh = min(n_frames, 100)
        hF = torch.stack([f.cpu() for f in frames[:nh]]).pin_memory()
        hS = torch.stack([s_.cpu() for s_ in src[:nh]]).pin_memory()
        hD = torch.stack([d_.cpu() for d_ in dst[:nh]]).pin_memory()
        e_steps = max(1, min(args.steps, 5))
        e_ms = []
        cstream = torch.cuda.Stream(device=dev)
        dF = [torch.empty((B,) + tuple(frames[0].shape), dtype=frames[0].dtype, device=dev)
              for _ in range(2)]
        dS = [torch.empty((B, n, 2), dtype=torch.float32, device=dev) for _ in range(2)]
        dD = [torch.empty((B, n, 2), dtype=torch.float32, device=dev) for _ in range(2)]
        h_infos = torch.empty((n_frames, 4), dtype=torch.int32).pin_memory()
        h_cs = torch.empty((n_frames, n), dtype=torch.float32).pin_memory()
        pos = {k: (i % 2, j) for i, ks in enumerate(batches) for j, k in enumerate(ks)}

        def e2e_step():
            m_ev, f_ev, free = {}, {}, {}

            def copy_in(i):
                sl = i % 2
                if sl in free:
                    cstream.wait_event(free[sl])
                with torch.cuda.stream(cstream):
                    for j0, h0, cnt in contiguous_runs(batches[i], nh):
                        dS[sl][j0:j0 + cnt].copy_(hS[h0:h0 + cnt], non_blocking=True)
                        dD[sl][j0:j0 + cnt].copy_(hD[h0:h0 + cnt], non_blocking=True)
                    m_ev[i] = torch.cuda.Event()
                    m_ev[i].record(cstream)
                    ks = batches[i]
                    for g0 in range(0, len(ks), G):
                        for j0, h0, cnt in contiguous_runs(ks[g0:g0 + G], nh):
                            dF[sl][g0 + j0:g0 + j0 + cnt].copy_(hF[h0:h0 + cnt], non_blocking=True)
                        f_ev[(i, g0 // G)] = torch.cuda.Event()
                        f_ev[(i, g0 // G)].record(cstream)

            def post(i):
                k0, cnt = batches[i][0], len(batches[i])
                h_infos[k0:k0 + cnt].copy_(infos[k0:k0 + cnt], non_blocking=True)
                h_cs[k0:k0 + cnt].copy_(c_all[i % nbuf, :cnt], non_blocking=True)
                free[i % 2] = torch.cuda.Event()
                free[i % 2].record(stream)
                if i + 2 < len(batches):
                    copy_in(i + 2)

            cstream.wait_stream(stream)
            for i in range(min(2, len(batches))):
                copy_in(i)
            fit_stream.wait_stream(stream)
            group_wait[0] = lambda i, g: stream.wait_event(f_ev[(i, g)])
            try:
                run_batches(batches, lambda k: dF[pos[k][0]][pos[k][1]], lambda k: dS[pos[k][0]][pos[k][1]],
                            lambda k: dD[pos[k][0]][pos[k][1]],
                            ready=lambda i, st: st.wait_event(m_ev[i]), post_blend=post)
            finally:
                group_wait[0] = None
            stream.wait_stream(cstream)

        # the step (copies in, calls, copies out) captured once into a CUDA graph like the
        # device pass, every replay copying the pinned host inputs again; direct calls if the
        # capture is refused
        e_graph, e_note = None, None
        if graph is not None:
            saved = (stream, fit_stream)
            try:
                cap = torch.cuda.Stream(device=dev)
                cap.wait_stream(torch.cuda.current_stream())
                g2 = torch.cuda.CUDAGraph()
                stream = fit_stream = cap
                with torch.cuda.graph(g2, stream=cap):
                    e2e_step()
                e_graph = g2
            except Exception as ex:
                e_note = f'capture failed, calls issued directly: {type(ex).__name__}: {ex}'[:300]
            stream, fit_stream = saved
            warm_done.clear()
            torch.cuda.synchronize()
        for i in range(1 + e_steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if e_graph is not None:
                e_graph.replay()
            else:
                e2e_step()
            b.record(stream)
            b.synchronize()
            if i >= 1:
                e_ms.append(a.elapsed_time(b))
        e_total = sum(e_ms)
        e_total = max_over_ranks(e_total, ws, dev)
        e2e = dict(value=job_mpix_per_s(ws, len(e_ms) * n_frames, sc.w, sc.h, e_total),
                   unit=UNIT, ms_per_frame=e_total / (len(e_ms) * n_frames),
                   h2d_bytes_per_step=int(n_frames * (frames[0].numel() + src[0].numel() * 8)),
                   d2h_bytes_per_step=int(n_frames * (16 + 4 * n)), cuda_graph=e_graph is not None,
                   **({'cuda_graph_note': e_note} if e_note else {}))

    # the plain FP32 GPU form of the same path, for the headline comparison: per frame
    # emdq_fit (no warm start) + the FP32 per-pixel field + warp, on 10 frames
    plain = None
    if not args.no_plain and rank == 0:
        fws = torch.empty(emdq.field_workspace_size(n, max_gw, max_gh, emdq.FP32), dtype=torch.uint8,
                          device=dev)
        cv2 = canvas.clone()
        pm = []
        for i in range(12):
            k = i % n_frames
            g = grids[k]
            disp = disp_buf[: g[2] * g[3] * 2].view(g[3], g[2], 2)
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = emdq.emdq_fit(src[k], dst[k], sc.w, sc.h, out=fit_outs_all[0][0], workspace=fit_ws_all[0])
            emdq.emdq_field(r['q'], r['c'], src[k], g, alpha, precision=emdq.FP32, out=disp, workspace=fws)
            emdq.mosaic_warp(frames[k], disp, g, cv2, origin)
            b.record(stream)
            b.synchronize()
            if i >= 2:
                pm.append(a.elapsed_time(b))
        plain = dict(value=sc.w * sc.h / 1e6 / (np.mean(pm) / 1e3), unit=UNIT,
                     ms_per_frame=float(np.mean(pm)), frames=len(pm),
                     path='emdq_fit + emdq_field (fp32 per-pixel) + mosaic_warp, one frame at a time')

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return None

    peaks = measured_peaks()
    win_px = float(np.mean([g[2] * g[3] for g in grids]))
    mean_iters = float(np.mean(iters))
    sm_mhz = (clk or {}).get('sm_mhz') or peaks['sm_max_mhz']
    alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    alu_src = f'derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x {sm_mhz:.0f} MHz (sampled SM clock)'
    # per-frame EM rounds of every fit launch (step-major, the order the events were taken)
    it_steps = [t[:, 1].cpu().numpy() for t in all_infos]
    launch_rounds = [float(np.sum(it_steps[i // len(batches)][fit_launch_frames[i]] + 1))
                     for i in range(len(fit_launch_frames))]
    kernel_total = dict(fit=float(np.sum(fit_ms)), warm=float(np.sum(warm_ms)),
                        field=float(np.sum(field_ms)), warp=float(np.sum(warp_ms)))
    if group_fused:
        # one call per group does both: its time is the field events' span
        kernel_total = dict(fit=kernel_total['fit'], warm=kernel_total['warm'],
                            mosaic=kernel_total['field'])
    dom = max(kernel_total, key=kernel_total.get)
    if dom == 'fit':
        # FP32 operations per match pair and EM round (an FMA counts 2): 34 in the M-step
        # pass, 22 in the leave-one-out blend
        flops = float(np.sum(launch_rounds)) * n * n * 56.0 / len(fit_ms)
        roof = dict(bound='alu', kernel=('emdq_fit_batch_kernel' + (' + emdq_fit_batch_next_kernel'
                                                                     if fit_sched['phases'] else '')
                                         if B > 1 else 'emdq_fit_kernel'),
                    achieved=flops / (np.mean(fit_ms) * 1e-3) / 1e12, peak=alu_peak, unit='TFLOP/s',
                    peak_source=alu_src, launches=len(fit_ms), mean_launch_ms=float(np.mean(fit_ms)),
                    work_per_launch=f'{flops:.4g} FP32 flops = 56 x EM rounds x N^2 over the '
                                    f'launch\'s {B} fits')
    elif dom == 'warm':
        # per match: N distance tests (4 flops) + the 16-64-64-1 network (2 x 5184 MACs)
        flops = B * n * (4.0 * n + 2 * 5184)
        roof = dict(bound='alu', kernel='warm_start_batch_kernel',
                    achieved=flops / (np.mean(warm_ms) * 1e-3) / 1e12, peak=alu_peak, unit='TFLOP/s',
                    peak_source=alu_src, launches=len(warm_ms), mean_launch_ms=float(np.mean(warm_ms)))
    elif dom in ('field', 'mosaic'):
        if prec == emdq.BF16:
            # the matches that carry weight (c > 0): zero-weight terms of Eqs. 2-3 are no work
            nz = []
            for bi, ks in enumerate(batches):
                fit_batch(bi, ks, lambda k: src[k], lambda k: dst[k])
                torch.cuda.synchronize()
                nz += [int((fit_outs_all[bi % nbuf][j]['c'] > 0).sum().item()) for j in range(len(ks))]
            flops = 2.0 * 6 * win_px * float(np.mean(nz))
            roof = dict(bound='tensor',
                        kernel=('emdq_mosaic_batch: field_tc_prep_kernel + mosaic_tc_kernel (the '
                                'field GEMM with the warp in its epilogue)'
                                if group_fused else
                                ('emdq_field_batch' if piped else 'emdq_field') +
                                ': field_tc_prep_kernel + field_tc_kernel') +
                               ' (timed together, per frame)',
                        work='2 x 6 x window pixels x matches of nonzero weight',
                        achieved=flops / (np.mean(field_ms) * 1e-3) / 1e12,
                        peak=peaks['bf16_tflops'], unit='TFLOP/s',
                        peak_source=peaks['source'] + ' bf16 burst', launches=len(field_ms),
                        mean_launch_ms=float(np.mean(field_ms)))
        else:
            flops = win_px * n * 17.0
            roof = dict(bound='alu', kernel='field_direct_kernel',
                        achieved=flops / (np.mean(field_ms) * 1e-3) / 1e12, peak=alu_peak,
                        unit='TFLOP/s', peak_source=alu_src, launches=len(field_ms),
                        mean_launch_ms=float(np.mean(field_ms)))
    else:
        nbytes = win_px * (8 + 8) + sc.w * sc.h * sc.channels
        roof = dict(bound='hbm', kernel='mosaic_warp_kernel',
                    achieved=nbytes / (np.mean(warp_ms) * 1e-3) / 1e9,
                    peak=peaks['hbm_gbs'], unit='GB/s', peak_source=peaks['source'] + ' copy',
                    launches=len(warp_ms), mean_launch_ms=float(np.mean(warp_ms)))
    roof['frac'] = roof['achieved'] / roof['peak']
    tr = NCU_TRAFFIC.get(dom if dom != 'field' or prec == emdq.BF16 else 'field_fp32')
    roof['traffic'] = tr['bytes'] if tr and tr['src'] == _src_hash(tr['file']) else None

    line = dict(
        metric=METRIC, value=job_mpix_per_s(ws, total_frames, sc.w, sc.h, total_ms), unit=UNIT,
        n_gpus=ws, steps=args.steps, warmup=args.warmup, ms_per_step=total_ms / args.steps,
        p50_frame_ms=float(np.median(frame_ms)), higher_is_better=True, scaling='weak',
        vs_baseline=None, dtype='bf16' if prec == emdq.BF16 else 'f32', data='synthetic',
        config=dict(workload_config(args, sc, cfg, n_frames, ws), precision=args.precision,
                    mean_window_px=win_px, mean_em_iters=mean_iters),
        kernel_ms_per_step={k: v / args.steps for k, v in kernel_total.items()},
        path=(('learned warm start + ' if warm else '') + ('emdq_fit_batch' if B > 1 else 'emdq_fit') +
              (f' in phases {fit_sched["phases"]} (emdq_fit_batch_phases)' if fit_sched['phases'] else '') +
              (' + emdq_mosaic (fused BF16 field and warp)' if fused else
               f' + emdq_mosaic_batch ({G} frames per call, bf16 field and warp fused)' if group_fused else
               (f' + emdq_field_batch + mosaic_warp_batch ({G} frames per call, bf16; ' +
                ('each call after the other on one stream)' if args.one_stream else
                 'the warps on a second stream)')
                if piped and prec == emdq.BF16 else f' + emdq_field ({args.precision}) + mosaic_warp')) +
              (', fits of the next batch on a second stream' if overlap else '') +
              (', warm starts one batch ahead on a third stream' if hoist else '') +
              (', the pass replayed from one CUDA graph' if graph is not None else '')),
        batch=B, field_group=G, field_autotune=field_tune, fit_schedule=fit_tune, warm_start=warm,
        cuda_graph=graph is not None,
        **({'cuda_graph_note': graph_note} if graph_note else {}), wall_s=wall, roofline=roof,
        gpu_launches=(args.steps * sum((2 if group_fused else 3) * ((len(ks) + G - 1) // G)
                                       for ks in batches) if G > 1 else
                      total_frames * (2 if fused else 3)) +
                     args.steps * len(batches) * ((2 if warm else 1) +
                                                  (len(fit_sched['phases']) - 1 if fit_sched['phases'] else 0)),
        clocks=clk,
        e2e=e2e, plain_fp32_gpu=plain, beside_the_step=unc,
        speedup_vs_plain_fp32_gpu=(None if plain is None else
                                   job_mpix_per_s(ws, total_frames, sc.w, sc.h, total_ms) / plain['value']),
        fit_status=statuses,
        canvas_sha256=hashlib.sha256(canvas.cpu().numpy().tobytes()).hexdigest()[:16],
    )
    if not args.no_cpu_baseline:
        line['cpu_baseline'] = cpu_baseline(args, budget_s=12.0)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return line


MIXED_COUNT = 64
MIXED_PAD = 256          # canvas margin around each pair's reference frame


def run_gpu_tiled(args, ws, rank, local):
    """`--shard canvas`: one sequence on W GPUs -- fits sharded by frame, one all-gather of the
    fit rows, field + warp of every frame on each rank's band of canvas rows (strong scaling)."""
    import numpy as np
    import torch
    import paper_2103_07414_gb300 as emdq
    from synth import WORKLOADS

    torch.cuda.set_device(local)
    dev = torch.device('cuda', local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=dev)
    n_frames = WORKLOADS[args.workload]['frames']
    if args.frames > 0:
        n_frames = min(n_frames, args.frames)
    sc, cfg, origin, ref, frames, src, dst, grids = prepare_sequence(args.workload, args.seed,
                                                                    n_frames, dev)
    cw, chh = cfg['canvas']
    n = cfg['n']
    band = canvas_band(chh, ws, rank)
    canvas = torch.zeros((chh, cw, 4), dtype=torch.uint8, device=dev)
    emdq.mosaic_insert_reference(ref, canvas, origin)
    alpha = emdq.alpha_for_frame(sc.w, sc.h)
    mine = list(range(rank, n_frames, ws))
    B = max(1, min(args.batch or cfg.get('batch', 50), 64))
    batches = [mine[i:i + B] for i in range(0, len(mine), B)]
    warm_params = emdq.load_warmstart_params(dev)
    outs = {k: dict(q=torch.empty((n, 8), device=dev), c=torch.empty(n, device=dev),
                    p=torch.empty(n, device=dev), info=torch.zeros(4, dtype=torch.int32, device=dev))
            for k in mine}
    p0 = {k: torch.empty(n, device=dev) for k in mine}
    fit_ws = torch.empty(max(256, emdq.fit_batch_workspace_size([(src[0], dst[0])] * B)),
                         dtype=torch.uint8, device=dev)
    clipped = [clip_to_band(g, origin, band) for g in grids]
    todo = [k for k in range(n_frames) if clipped[k] is not None]
    G = max(1, min(8, args.field_group or 4))
    groups = [todo[i:i + G] for i in range(0, len(todo), G)]
    zq, zc, zs = torch.zeros((n, 8), device=dev), torch.zeros(n, device=dev), torch.zeros((n, 2), device=dev)
    gw_max = max([clipped[k][2] for k in todo] + [1])
    gh_max = max([clipped[k][3] for k in todo] + [1])
    gws = torch.empty(emdq.field_batch_workspace_size([(zq, zc, zs, (0, 0, gw_max, gh_max), alpha)] * G),
                      dtype=torch.uint8, device=dev)
    disp = [torch.empty(gw_max * gh_max * 2, device=dev) for _ in range(G)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def one_pass():
        for ks in batches:
            emdq.warm_start([(src[k], dst[k]) for k in ks], warm_params, outs=[p0[k] for k in ks])
            emdq.emdq_fit_batch([(src[k], dst[k], sc.w, sc.h, p0[k]) for k in ks],
                                outs=[outs[k] for k in ks], workspace=fit_ws)
        rows = {k: torch.cat([outs[k]['q'], outs[k]['c'][:, None]], 1) for k in mine}
        allrows = gather_fit_rows(rows, ws, rank, n_frames, n, dev)
        for grp in groups:
            ds = [disp[i][: clipped[k][2] * clipped[k][3] * 2].view(clipped[k][3], clipped[k][2], 2)
                  for i, k in enumerate(grp)]
            emdq.emdq_field_batch([(allrows[k][:, :8].contiguous(), allrows[k][:, 8].contiguous(), src[k],
                                    clipped[k], alpha) for k in grp], outs=ds, workspace=gws)
            emdq.mosaic_warp_batch([frames[k] for k in grp], ds, [clipped[k] for k in grp], canvas, origin)

    t0 = time.perf_counter()
    w = 0
    while w < args.warmup or time.perf_counter() - t0 < args.min_warmup_s:
        flush.zero_()
        one_pass()
        torch.cuda.synchronize()
        w += 1
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.1)
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        one_pass()
        b.record()
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(float(np.sum(step_ms)), ws, dev)
    digest = hashlib.sha256(canvas[band[0]:band[1]].cpu().numpy().tobytes()).hexdigest()[:16]
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return None
    value = args.steps * n_frames * sc.w * sc.h / 1e6 / (total_ms / 1e3)
    cfgd = workload_config(args, sc, cfg, n_frames, ws)
    cfgd['parallelism'] = f'canvas bands x{ws}: fits sharded by frame, one all-gather of the fit rows per pass'
    return dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps,
                warmup=args.warmup, ms_per_step=total_ms / args.steps,
                p50_frame_ms=float(np.median(step_ms)) / n_frames, higher_is_better=True,
                scaling='strong', vs_baseline=None, dtype='bf16', data='synthetic', config=cfgd,
                path='per rank: warm start + emdq_fit_batch on frames k = rank mod W, all-gather of '
                     'the fit rows, emdq_field_batch + mosaic_warp_batch of every frame on the '
                     "rank's band of canvas rows, frames in order",
                gpu_launches=args.steps * (2 * len(batches) + 3 * len(groups)), clocks=clk, e2e=None,
                band0_sha256=digest)


def mixed_config(args, ws, pairs, ctas=None) -> dict:
    sizes = sorted({(p['scene'].w, p['scene'].h) for p in pairs})
    ns = [p['n'] for p in pairs]
    cfg = dict(workload=f'batch64: {len(pairs)} independent frame pairs, sizes uniform over '
                        f'{{640x480, 1280x720, 1280x1024, 1920x1080}} RGB8, N uniform in [100, 3000], '
                        f'outliers uniform in [10%, 40%]; one step = every pair through warm start, '
                        f'fit, field and warp (each pair into its own canvas)',
               pairs=len(pairs), sizes_present=[f'{w}x{h}' for w, h in sizes],
               n_min=min(ns), n_max=max(ns), n_mean=float(sum(ns)) / len(ns),
               frame_pixels_per_step=int(sum(p['scene'].w * p['scene'].h for p in pairs)),
               parallelism=f'dp{ws} (independent batches)',
               l2='inputs larger than L2 (64 distinct frames) and a 256 MiB flush before every '
                  'step, outside the timed events')
    if ctas is not None:
        cfg['fit_ctas_autotuned'] = ctas
    return cfg


def run_gpu_mixed(args, ws, rank, local):
    """The mixed-size batch: 64 independent pairs per step, one warm-start launch, one
    autotuned fit launch (or the fits in phases), then the fields and warps of 16 pairs per
    emdq_mosaic_pairs call (--split-pairs: emdq_field_batch + mosaic_warp), the whole step one
    CUDA graph."""
    import numpy as np
    import torch
    import paper_2103_07414_gb300 as emdq
    from synth import canvas_origin, footprint_window, mixed_pairs, render_frame, render_reference

    torch.cuda.set_device(local)
    dev = torch.device('cuda', local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=dev)
    pairs = mixed_pairs(rank_seed(args.seed, rank), MIXED_COUNT)
    P = []
    for p in pairs:
        sc = p['scene']
        cw, chh = sc.w + 2 * MIXED_PAD, sc.h + 2 * MIXED_PAD
        origin = canvas_origin(cw, chh, sc.w, sc.h)
        canvas = torch.zeros((chh, cw, 4), dtype=torch.uint8, device=dev)
        emdq.mosaic_insert_reference(render_reference(sc, device=dev), canvas, origin)
        n = p['n']
        P.append(dict(sc=sc, n=n, origin=origin, canvas=canvas, grid=footprint_window(sc, 1, cw, chh),
                      frame=render_frame(sc, 1, device=dev), src=torch.from_numpy(p['src']).to(dev),
                      dst=torch.from_numpy(p['dst']).to(dev), alpha=emdq.alpha_for_frame(sc.w, sc.h),
                      out=dict(q=torch.empty((n, 8), device=dev), c=torch.empty(n, device=dev),
                               p=torch.empty(n, device=dev),
                               info=torch.zeros(4, dtype=torch.int32, device=dev)),
                      p0=torch.empty(n, device=dev)))
    warm_params = emdq.load_warmstart_params(dev)
    probs_sd = [(x['src'], x['dst']) for x in P]
    fit_probs = [(x['src'], x['dst'], x['sc'].w, x['sc'].h, x['p0']) for x in P]
    batch_ws = torch.empty(emdq.fit_batch_workspace_size(probs_sd), dtype=torch.uint8, device=dev)
    field_ws = torch.empty(max(emdq.field_workspace_size(x['n'], x['grid'][2], x['grid'][3], emdq.BF16)
                               for x in P), dtype=torch.uint8, device=dev)
    disp_buf = torch.empty(max(x['grid'][2] * x['grid'][3] for x in P) * 2, dtype=torch.float32,
                           device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    infos = torch.zeros((len(P), 4), dtype=torch.int32, device=dev)
    emdq.warm_start(probs_sd, warm_params, outs=[x['p0'] for x in P])
    ctas, tune_ms = emdq.fit_batch_autotune(fit_probs, reps=2, outs=[x['out'] for x in P],
                                            workspace=batch_ws)
    # then one launch with that split, or the batch in phases (the rounds of the autotuner's runs)
    fit_phases, fit_tune = None, None
    if not args.no_fit_phases:
        its = [int(x['out']['info'][1].item()) for x in P]
        fit_phases, ms = tune_fit_phases(emdq, [(fit_probs, [x['out'] for x in P], batch_ws, ctas)], its)
        fit_tune = dict(chosen='one launch (autotuned split)' if fit_phases is None else fit_phases,
                        ms_per_launch=ms)

    # fused (default): the fields and warps of a group of up to 16 pairs in one
    # emdq_mosaic_pairs call; split: the fields of a group of G pairs in one emdq_field_batch
    # call (main stream), their warps on the warp stream beside the next group's fields,
    # buffers double-buffered
    fused = not args.split_pairs
    G = max(1, min(16, args.field_group or (16 if fused else 4)))
    warp_stream = torch.cuda.Stream(device=dev)
    groups = [list(range(b0, min(len(P), b0 + G))) for b0 in range(0, len(P), G)]

    def pair_args(b):
        x = P[b]
        return (x['out']['q'], x['out']['c'], x['src'], x['grid'], x['alpha'], x['frame'], x['canvas'],
                x['origin'])

    if fused:
        gws = max(emdq.mosaic_pairs_workspace_size([pair_args(b) for b in grp]) for grp in groups)
    else:
        gws = max(emdq.field_batch_workspace_size([(P[b]['out']['q'], P[b]['out']['c'], P[b]['src'],
                                                    P[b]['grid'], P[b]['alpha']) for b in grp])
                  for grp in groups)
    grp_ws = [torch.empty(gws, dtype=torch.uint8, device=dev) for _ in range(2)]
    max_px = max(x['grid'][2] * x['grid'][3] for x in P)
    grp_disp = [] if fused else [[torch.empty(max_px * 2, dtype=torch.float32, device=dev) for _ in range(G)]
                                 for _ in range(2)]

    def one_pass(ev=None):
        # ev[0] start, ev[1] warm start done, ev[2] fits done, then fused: ev[3 + g] group g's
        # call done; split: per pair b ev[3 + 3b] field done (its group's call), ev[4 + 3b] /
        # ev[5 + 3b] warp start / done
        main = torch.cuda.current_stream()
        if ev: ev[0].record()
        emdq.warm_start(probs_sd, warm_params, outs=[x['p0'] for x in P])
        if ev: ev[1].record()
        emdq.emdq_fit_batch(fit_probs, outs=[x['out'] for x in P], workspace=batch_ws,
                            ctas=ctas if fit_phases is None else None, phases=fit_phases)
        if ev: ev[2].record()
        if fused:
            for gi, grp in enumerate(groups):
                emdq.emdq_mosaic_pairs([pair_args(b) for b in grp], workspace=grp_ws[0])
                if ev: ev[3 + gi].record(main)
            for b, x in enumerate(P):
                infos[b].copy_(x['out']['info'])
            return
        free = [None, None]
        for gi, grp in enumerate(groups):
            slot = gi % 2
            if free[slot] is not None:
                main.wait_event(free[slot])
            disps = [grp_disp[slot][i][: P[b]['grid'][2] * P[b]['grid'][3] * 2].view(
                     P[b]['grid'][3], P[b]['grid'][2], 2) for i, b in enumerate(grp)]
            emdq.emdq_field_batch([(P[b]['out']['q'], P[b]['out']['c'], P[b]['src'], P[b]['grid'],
                                    P[b]['alpha']) for b in grp], outs=disps, workspace=grp_ws[slot])
            fdone = torch.cuda.Event()
            fdone.record(main)
            if ev:
                for b in grp: ev[3 + 3 * b].record(main)
            warp_stream.wait_event(fdone)
            for i, b in enumerate(grp):
                x = P[b]
                if ev: ev[4 + 3 * b].record(warp_stream)
                emdq.mosaic_warp(x['frame'], disps[i], x['grid'], x['canvas'], x['origin'], stream=warp_stream)
                if ev: ev[5 + 3 * b].record(warp_stream)
            wdone = torch.cuda.Event()
            wdone.record(warp_stream)
            free[slot] = wdone
        main.wait_stream(warp_stream)
        for b, x in enumerate(P):
            infos[b].copy_(x['out']['info'])

    t0 = time.perf_counter()
    w = 0
    while w < args.warmup or time.perf_counter() - t0 < args.min_warmup_s:
        flush.zero_()
        one_pass()
        torch.cuda.synchronize()
        w += 1
    # the field tile height of every group, chosen by the library's autotuner (recorded per
    # size class, so the step's emdq_field_batch calls use it; the fused calls take 40 rows)
    field_tiles = []
    for grp in ([] if fused else groups):
        disps = [grp_disp[0][i][: P[b]['grid'][2] * P[b]['grid'][3] * 2].view(
                 P[b]['grid'][3], P[b]['grid'][2], 2) for i, b in enumerate(grp)]
        py, _ = emdq.field_batch_autotune([(P[b]['out']['q'], P[b]['out']['c'], P[b]['src'], P[b]['grid'],
                                            P[b]['alpha']) for b in grp], reps=3, outs=disps,
                                          workspace=grp_ws[0])
        field_tiles.append(py)
    field_tiles = [40] * len(groups) if fused else [
        emdq.field_batch_tile_rows([(P[b]['out']['q'], P[b]['out']['c'], P[b]['src'], P[b]['grid'],
                                     P[b]['alpha']) for b in grp]) for grp in groups]
    n_ev = 3 + (len(groups) if fused else 3 * len(P))
    graph, graph_note = None, None
    gev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(n_ev)]
    if not args.no_graph:
        try:
            cap = torch.cuda.Stream(device=dev)
            cap.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                one_pass(gev)
            graph = g
        except Exception as ex:
            graph_note = f'capture failed, calls issued directly: {type(ex).__name__}: {ex}'[:300]
        torch.cuda.synchronize()
    warm_ms, fit_ms, field_ms, warp_ms, mosaic_ms, step_ms = [], [], [], [], [], []

    def collect(ev):
        warm_ms.append(ev[0].elapsed_time(ev[1]))
        fit_ms.append(ev[1].elapsed_time(ev[2]))
        prev = ev[2]
        if fused:
            for gi in range(len(groups)):
                mosaic_ms.append(prev.elapsed_time(ev[3 + gi]))
                prev = ev[3 + gi]
            return
        for b in range(len(P)):
            field_ms.append(prev.elapsed_time(ev[3 + 3 * b]))
            warp_ms.append(ev[4 + 3 * b].elapsed_time(ev[5 + 3 * b]))
            prev = ev[3 + 3 * b]

    outer = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.steps)]
    direct_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.1)
    all_infos = []
    for i in range(args.steps):
        flush.zero_()
        outer[i][0].record()
        if graph is not None:
            graph.replay()
        else:
            one_pass(direct_ev[i])
        outer[i][1].record()
        outer[i][1].synchronize()
        collect(gev if graph is not None else direct_ev[i])
        step_ms.append(outer[i][0].elapsed_time(outer[i][1]))
        all_infos.append(infos.clone())
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(float(np.sum(step_ms)), ws, dev)
    px = sum(x['sc'].w * x['sc'].h for x in P)
    iv = torch.stack(all_infos).cpu()
    iters = iv[:, :, 1].numpy()
    statuses = sorted({emdq.STATUS.get(int(v), '?') for v in iv[:, :, 0].flatten().tolist()})
    nz = [int((x['out']['c'] > 0).sum().item()) for x in P]
    # end to end through the single public call: per step the H2D copy of every pair's frame
    # and matches from pinned host buffers, emdq_batch (warm start, fits, fields, warps on one
    # stream), and the D2H of the fit records and field weights; its device time without the
    # copies is reported beside it
    e2e, native_ms = None, None
    if not args.no_e2e:
        pairs_native = [dict(src=x['src'], dst=x['dst'], frame=x['frame'], grid=x['grid'],
                             canvas=x['canvas'], origin=x['origin']) for x in P]
        bws = torch.empty(emdq.batch_workspace_size(pairs_native, warm=True), dtype=torch.uint8, device=dev)
        hf = [x['frame'].cpu().pin_memory() for x in P]
        hs = [x['src'].cpu().pin_memory() for x in P]
        hd = [x['dst'].cpu().pin_memory() for x in P]
        h_infos = torch.empty((len(P), 4), dtype=torch.int32).pin_memory()
        h_cs = [torch.empty(x['n'], dtype=torch.float32).pin_memory() for x in P]
        outs = [x['out'] for x in P]
        e_steps = max(1, min(args.steps, 5))
        e_ms, n_ms = [], []
        main = torch.cuda.current_stream()
        for i in range(2 * (1 + e_steps)):
            copies = i % 2 == 0
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main)
            if copies:
                for k, x in enumerate(P):
                    x['frame'].copy_(hf[k], non_blocking=True)
                    x['src'].copy_(hs[k], non_blocking=True)
                    x['dst'].copy_(hd[k], non_blocking=True)
            emdq.emdq_batch(pairs_native, warm_params=warm_params, outs=outs, workspace=bws,
                            fit_ctas=ctas if fit_phases is None else None, fit_phases=fit_phases)
            if copies:
                for k, x in enumerate(P):
                    infos[k].copy_(x['out']['info'])
                    h_cs[k].copy_(x['out']['c'], non_blocking=True)
                h_infos.copy_(infos, non_blocking=True)
            b.record(main)
            b.synchronize()
            if i >= 2:
                (e_ms if copies else n_ms).append(a.elapsed_time(b))
        e_total = max_over_ranks(float(np.sum(e_ms)), ws, dev)
        native_ms = max_over_ranks(float(np.mean(n_ms)), ws, dev)
        px_all = sum(x['sc'].w * x['sc'].h for x in P)
        e2e = dict(value=ws * len(e_ms) * px_all / 1e6 / (e_total / 1e3), unit=UNIT,
                   call='emdq_batch', ms_per_step=e_total / len(e_ms),
                   h2d_bytes_per_step=int(sum(x['frame'].numel() + x['src'].numel() * 8 for x in P)),
                   d2h_bytes_per_step=int(sum(16 + 4 * x['n'] for x in P)))

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return None
    peaks = measured_peaks()
    sm_mhz = (clk or {}).get('sm_mhz') or peaks['sm_max_mhz']
    alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    totals = dict(fit=float(np.sum(fit_ms)), warm=float(np.sum(warm_ms)))
    if fused:
        totals['mosaic'] = float(np.sum(mosaic_ms))
    else:
        totals.update(field=float(np.sum(field_ms)), warp=float(np.sum(warp_ms)))
    dom = max(totals, key=totals.get)
    ns = np.array([x['n'] for x in P], dtype=np.float64)
    win = np.array([x['grid'][2] * x['grid'][3] for x in P], dtype=np.float64)
    if dom == 'fit':
        flops = float(np.mean([np.sum((it + 1) * ns * ns) for it in iters])) * 56.0
        roof = dict(bound='alu', kernel='emdq_fit_batch_kernel' + (' + emdq_fit_batch_next_kernel'
                                                                    if fit_phases else ''), achieved=flops / (np.mean(fit_ms) * 1e-3) / 1e12,
                    peak=alu_peak, unit='TFLOP/s',
                    peak_source=f'derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x {sm_mhz:.0f} MHz',
                    launches=len(fit_ms), mean_launch_ms=float(np.mean(fit_ms)))
    elif dom == 'field':
        flops = 2.0 * 6 * float(np.sum(win * np.array(nz)))
        roof = dict(bound='tensor', kernel='emdq_field_batch: field_tc_prep_kernel + field_tc_kernel',
                    achieved=flops / (np.sum(field_ms) / args.steps * 1e-3) / 1e12,
                    peak=peaks['bf16_tflops'], unit='TFLOP/s', peak_source=peaks['source'] + ' bf16 burst',
                    launches=len(field_ms), mean_launch_ms=float(np.mean(field_ms)),
                    work='2 x 6 x window pixels x matches of nonzero weight, summed over the pairs')
    elif dom == 'mosaic':
        flops = 2.0 * 6 * float(np.sum(win * np.array(nz)))
        roof = dict(bound='tensor', kernel='emdq_mosaic_pairs: field_tc_prep_kernel + mosaic_tc_kernel (pairs)',
                    achieved=flops / (np.sum(mosaic_ms) / args.steps * 1e-3) / 1e12,
                    peak=peaks['bf16_tflops'], unit='TFLOP/s', peak_source=peaks['source'] + ' bf16 burst',
                    launches=len(mosaic_ms), mean_launch_ms=float(np.mean(mosaic_ms)),
                    work='2 x 6 x window pixels x matches of nonzero weight, summed over the pairs '
                         '(the warp and blend in the epilogue are not counted as work)')
    elif dom == 'warm':
        flops = float(np.sum(ns * (4.0 * ns + 2 * 5184)))
        roof = dict(bound='alu', kernel='warm_start_batch_kernel', achieved=flops / (np.mean(warm_ms) * 1e-3) / 1e12,
                    peak=alu_peak, unit='TFLOP/s', peak_source='derived', launches=len(warm_ms),
                    mean_launch_ms=float(np.mean(warm_ms)))
    else:
        nbytes = float(np.sum(win * 16 + np.array([x['sc'].w * x['sc'].h * 3 for x in P])))
        roof = dict(bound='hbm', kernel='mosaic_warp_kernel',
                    achieved=nbytes / (np.sum(warp_ms) / args.steps * 1e-3) / 1e9, peak=peaks['hbm_gbs'],
                    unit='GB/s', peak_source=peaks['source'] + ' copy', launches=len(warp_ms),
                    mean_launch_ms=float(np.mean(warp_ms)))
    roof['frac'] = roof['achieved'] / roof['peak']
    roof['traffic'] = None
    value = ws * args.steps * px / 1e6 / (total_ms / 1e3)
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps, warmup=args.warmup,
        ms_per_step=total_ms / args.steps, p50_frame_ms=float(np.median(step_ms)),
        higher_is_better=True, scaling='weak', vs_baseline=None, dtype='bf16', data='synthetic',
        config=mixed_config(args, ws, pairs, ctas),
        kernel_ms_per_step={k: v / args.steps for k, v in totals.items()},
        path='learned warm start (one launch) + ' +
             ('emdq_fit_batch (one launch, autotuned CTA split)' if fit_phases is None else
              f'emdq_fit_batch in phases {fit_phases} (emdq_fit_batch_phases)') + ' + ' +
             (f'emdq_mosaic_pairs ({G} pairs per call, bf16 field and warp fused)' if fused else
              f'emdq_field_batch ({G} pairs per call, bf16), their mosaic_warp on a second stream') +
             (', the step replayed from one CUDA graph' if graph is not None else ''),
        cuda_graph=graph is not None, **({'cuda_graph_note': graph_note} if graph_note else {}),
        autotune_fit_ms=tune_ms, fit_schedule=fit_tune, field_tile_rows=field_tiles,
        mean_em_iters=float(np.mean(iters)),
        roofline=roof,
        gpu_launches=args.steps * (2 + (len(fit_phases) - 1 if fit_phases else 0) + 2 * len(groups) +
                                   (0 if fused else len(P))),
        clocks=clk, e2e=e2e, fit_status=statuses,
        emdq_batch_device_ms=native_ms,
        p50_note='per step: the whole batch of 64 pairs is one unit of latency')
    if not args.no_cpu_baseline:
        line['cpu_baseline'] = cpu_baseline_mixed(args, budget_s=12.0)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return line


def oracle_pair(orc, p, frac):
    """One mixed pair through the oracle: the full fit, field and warp on a centred band of
    `frac` of the window's rows.  Returns seconds extrapolated to the whole window."""
    import numpy as np
    from synth import canvas_origin, footprint_window, render_frame
    sc = p['scene']
    cw, chh = sc.w + 2 * MIXED_PAD, sc.h + 2 * MIXED_PAD
    origin = canvas_origin(cw, chh, sc.w, sc.h)
    grid = footprint_window(sc, 1, cw, chh)
    canvas = np.zeros((chh, cw, 4), np.uint8)
    fr = render_frame(sc, 1).numpy()
    s = np.float32(p['src']).astype(np.float64)
    d = np.float32(p['dst']).astype(np.float64)
    t0 = time.perf_counter()
    r = orc.fit(s, d, sc.w, sc.h)
    t1 = time.perf_counter()
    rows = max(1, int(round(grid[3] * frac)))
    band = (grid[0], grid[1] + (grid[3] - rows) // 2, grid[2], rows)
    disp = orc.field(r['q8'], r['c'], s, band, orc.alpha_for_frame(sc.w, sc.h))
    orc.warp(fr, disp.astype(np.float32), band, canvas, origin)
    t2 = time.perf_counter()
    return (t1 - t0) + (t2 - t1) * grid[3] / rows


def cpu_baseline_mixed(args, budget_s=12.0):
    """The oracle on this host's cores over the first pairs of the batch (bounded sample)."""
    import oracle as orc
    from synth import mixed_pairs
    orc.build()
    pairs = mixed_pairs(args.seed, MIXED_COUNT)
    t_start, sec, px, k = time.perf_counter(), 0.0, 0, 0
    while k < len(pairs) and (time.perf_counter() - t_start < budget_s or k == 0):
        sec += oracle_pair(orc, pairs[k], 1.0)
        px += pairs[k]['scene'].w * pairs[k]['scene'].h
        k += 1
    return dict(value=px / 1e6 / sec, unit=UNIT, cores=orc.max_threads(), kind='oracle',
                sample=f'the first {k} pair(s) of the batch: full EM fit + field and warp over '
                       f'the whole window')


def run_reference_mixed(args, ws, rank):
    """--impl reference on the mixed batch: the oracle on the host cores, rank 0 only."""
    if rank != 0:
        return None
    import numpy as np
    import oracle as orc
    from synth import mixed_pairs
    orc.build()
    pairs = mixed_pairs(args.seed, MIXED_COUNT)
    times, pxs = [], []
    for k in range(args.warmup + args.steps):
        p = pairs[k % len(pairs)]
        t = oracle_pair(orc, p, 1.0)
        if k >= args.warmup:
            times.append(t)
            pxs.append(p['scene'].w * p['scene'].h)
    value = float(np.sum(pxs)) / 1e6 / float(np.sum(times))
    return dict(impl='reference', metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps,
                warmup=args.warmup, ms_per_step=float(np.mean(times)) * 1e3,
                p50_frame_ms=float(np.median(times)) * 1e3, higher_is_better=True, scaling='weak',
                vs_baseline=None, dtype='f64', data='synthetic',
                config=dict(mixed_config(args, ws, pairs), precision='f64',
                            sample='per step one pair of the batch: full EM fit + field and warp over '
                                   'the whole window'),
                cpu_baseline=dict(value=value, unit=UNIT, cores=orc.max_threads(), kind='oracle',
                                  sample='per step one pair of the batch, whole window'),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))


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
    frac = 1.0              # whole windows, as the reference arm samples them
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
                sample=f'{frames} frame(s) of the sequence: full EM fit + field and warp over '
                       f'the whole window',
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
                config=dict(workload_config(args, sc, cfg, cfg['frames'], ws), precision='f64',
                            sample=f'per step one frame of the sequence: full EM fit + field and '
                                   f'warp on {frac:.3f} of the window rows, extrapolated'),
                cpu_baseline=dict(value=value, unit=UNIT, cores=orc.max_threads(), kind='oracle',
                                  sample=f'per step: full EM fit + field and warp on {frac:.3f} of '
                                         f'the window rows, extrapolated to the full window'),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))


SUB_KEYS = ('value', 'unit', 'ms_per_step', 'p50_frame_ms', 'dtype', 'config', 'path', 'fit_schedule',
            'kernel_ms_per_step', 'roofline', 'cpu_baseline', 'e2e', 'clocks', 'fit_status',
            'mean_em_iters', 'gpu_launches', 'steps', 'warmup', 'p50_note', 'field_autotune',
            'field_tile_rows')


def sub_result(line: dict) -> dict:
    return {k: line[k] for k in SUB_KEYS if k in line and line[k] is not None}


def extras(args, local) -> dict:
    """Results printed beside the default line (one GPU): the latency mode of the same
    sequence (one frame in flight: warm start, fit, fused BF16 field and warp per frame), the
    64-pair mixed batch and the 500-frame 1920x1080 sequence, each with its roofline object
    and its own bounded oracle sample."""
    import copy
    import torch
    out = {}

    def sub(**kw):
        a = copy.copy(args)
        a.no_e2e, a.no_plain, a.no_beside, a.frames = True, True, True, 0
        a.min_warmup_s = 0.2
        for k, v in kw.items():
            setattr(a, k, v)
        return a

    lat = run_gpu(sub(batch=1, field_group=1, steps=min(args.steps, 5), no_cpu_baseline=True), 1, 0, local)
    out['latency_mode'] = dict(
        sub_result(lat), mode='one frame in flight: per frame the learned warm start, emdq_fit and one '
                              'fused BF16 field and warp (emdq_mosaic_batch of one frame)',
        ms_per_frame=lat['ms_per_step'] / lat['config']['frames_per_step'])
    torch.cuda.empty_cache()
    out['batch64'] = sub_result(run_gpu_mixed(sub(workload='batch64', steps=min(args.steps, 10)), 1, 0, local))
    torch.cuda.empty_cache()
    out['seq1920'] = sub_result(run_gpu(sub(workload='seq1920', steps=2, batch=0), 1, 0, local))
    torch.cuda.empty_cache()
    return out


def main():
    args = parse_args()
    ws, rank, local = dist_env()
    mixed = args.workload == 'batch64'
    if args.impl == 'reference':
        line = run_reference_mixed(args, ws, rank) if mixed else run_reference(args, ws, rank)
    else:
        if mixed:
            line = run_gpu_mixed(args, ws, rank, local)
        elif args.shard == 'canvas':
            line = run_gpu_tiled(args, ws, rank, local)
        else:
            line = run_gpu(args, ws, rank, local)
        if (line is not None and ws == 1 and args.workload == 'seq1280' and args.shard == 'sequence'
                and not args.no_extras and args.frames == 0):
            ex = extras(args, local)
            line['latency_mode'] = ex.pop('latency_mode')
            line['other_workloads'] = ex
    if line is not None and rank == 0:
        print(json.dumps(line))


if __name__ == '__main__':
    main()
