"""World-size-2 gloo test (CPU) of the multi-rank benchmark path: per-rank sequences,
barrier, max-over-ranks timing and the whole-job throughput; the reference arm runs on
rank 0 only."""
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
