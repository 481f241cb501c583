"""World-size-2 gloo tests (CPU) of the multi-rank benchmark paths: per-rank sequences,
barrier, max-over-ranks timing and the whole-job throughput; one sequence split into canvas
bands with the fits sharded by frame and gathered; the reference arm runs on rank 0 only."""
import json
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_shard_by_sequence(tmp_path, orc):
    import torch.multiprocessing as mp

    from multirank_worker import worker
    fake_ms = [120.0, 150.0]
    mp.start_processes(worker, args=(2, _free_port(), str(tmp_path), fake_ms), nprocs=2,
                       join=True, start_method='spawn')
    r = [json.load(open(tmp_path / f'rank{k}.json')) for k in range(2)]
    # independent problems: different seeds, different matches
    assert r[0]['seed'] != r[1]['seed']
    assert r[0]['first'][0] != r[0]['first'][1]
    assert r[0]['first'] == r[1]['first']              # both ranks saw the same gather
    # the job's time is the slowest rank's, on every rank
    assert r[0]['t_max'] == r[1]['t_max'] == max(fake_ms)
    # whole-job throughput: all ranks' pixels over that time
    assert r[0]['value'] == pytest.approx(2 * 100 * 640 * 480 / 1e6 / 0.150)
    # each rank's fit is complete on its own
    for x in r:
        assert x['precision'] >= 0.95 and x['recall'] >= 0.95


def test_max_over_ranks_is_identity_on_one_rank():
    import bench
    assert bench.max_over_ranks(3.25, 1, None) == 3.25
    assert bench.job_mpix_per_s(1, 10, 1000, 1000, 1000.0) == pytest.approx(10.0)
    assert bench.rank_seed(5, 0) == 5 and bench.rank_seed(5, 1) != bench.rank_seed(5, 0)


def test_reference_arm_runs_on_rank_zero_only():
    import bench
    # the other ranks return at once, without work (and without reading any argument)
    assert bench.run_reference(None, 2, 1) is None


def test_two_gloo_ranks_split_one_sequence_into_canvas_bands(tmp_path, orc):
    import numpy as np
    import torch.multiprocessing as mp

    from multirank_worker import tiled_worker
    from synth import canvas_origin, footprint_window, make_matches, workload
    n_frames = 5                                        # ragged: rank 0 fits 3, rank 1 fits 2
    mp.start_processes(tiled_worker, args=(2, _free_port(), str(tmp_path), n_frames), nprocs=2,
                       join=True, start_method='spawn')
    rows = [np.load(tmp_path / f'rows{k}.npy') for k in range(2)]
    tiles = [json.load(open(tmp_path / f'tiles{k}.json')) for k in range(2)]
    assert tiles[0]['owned'] == [0, 2, 4] and tiles[1]['owned'] == [1, 3]
    # after the all-gather both ranks hold every frame's fit rows, in frame order, equal to a
    # fit of that frame on one rank
    np.testing.assert_array_equal(rows[0], rows[1])
    sc, cfg = workload('pair640', seed=4)
    for k in (0, 3):
        s, d, _ = make_matches(sc, 1 + k, cfg['n'], cfg['outliers'], cfg['noise'])
        f = orc.fit(np.float32(s).astype(np.float64), np.float32(d).astype(np.float64), sc.w, sc.h)
        want = np.concatenate([f['q8'], f['c'][:, None]], 1).astype(np.float32)
        np.testing.assert_array_equal(rows[0][k], want)
    # the bands tile the canvas rows exactly once; each frame's window rows split between them
    cw, chh = cfg['canvas']
    assert tiles[0]['band'][0] == 0 and tiles[0]['band'][1] == tiles[1]['band'][0]
    assert tiles[1]['band'][1] == chh
    origin = canvas_origin(cw, chh, sc.w, sc.h)
    for k in range(n_frames):
        g = footprint_window(sc, 1 + k, cw, chh)
        parts = [t['clips'][k] for t in tiles if t['clips'][k] is not None]
        assert sum(p[3] for p in parts) == g[3]
        assert all(p[0] == g[0] and p[2] == g[2] for p in parts)
        ys = sorted((p[1], p[1] + p[3]) for p in parts)
        assert ys[0][0] == g[1] and ys[-1][1] == g[1] + g[3]
        assert all(a[1] == b[0] for a, b in zip(ys, ys[1:]))
        for t, p in zip(tiles, [t['clips'][k] for t in tiles]):
            if p is not None:
                assert t['band'][0] <= p[1] + origin[1] and p[1] + p[3] + origin[1] <= t['band'][1]


def test_contiguous_runs_of_host_rows():
    """The end-to-end leg copies a batch's frames in runs of consecutive host rows k % nh:
    one run when the batch does not wrap, two when it crosses a multiple of nh, every frame
    exactly once and in batch order."""
    import bench
    assert bench.contiguous_runs(list(range(50, 100)), 100) == [(0, 50, 50)]
    assert bench.contiguous_runs(list(range(96, 104)), 100) == [(0, 96, 4), (4, 0, 4)]
    assert bench.contiguous_runs([7], 16) == [(0, 7, 1)]
    for ks, nh in ((list(range(0, 64)), 16), (list(range(13, 77)), 20), (list(range(99, 101)), 100)):
        runs = bench.contiguous_runs(ks, nh)
        rows = [h + i for _, h, c in runs for i in range(c)]
        slots = [j + i for j, _, c in runs for i in range(c)]
        assert rows == [k % nh for k in ks] and slots == list(range(len(ks)))
