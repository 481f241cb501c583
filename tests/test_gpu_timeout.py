"""The fit's bounded device-side waits end: a fit whose grid barriers cannot be passed (the
test setting emdq_params.reserved[1] makes every barrier wait for one arrival more than the
grid makes) returns with EMDQ_ETIMEOUT in its info record once each CTA's wait reaches its
bound, and the context stays usable: the next fit on the same stream and workspace gives
the same bits as a fit that never saw a timeout.  Nothing here faults or hangs: every wait is
bounded (reserved[0] lowers the bound to a few thousand polls; the default, about half a
second of polling, is taken once)."""
import time

import pytest
import torch

from synth import make_matches, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _matches(name, seed, t=1):
    sc, cfg = workload(name, seed=seed)
    src, dst, _ = make_matches(sc, t, cfg['n'], cfg['outliers'], cfg['noise'])
    return sc, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()


def _timed(fn):
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1), time.perf_counter() - t0


@pytest.mark.parametrize('polls', [5000, 0])      # a lowered bound, then the default one
def test_unreachable_barrier_times_out_and_the_next_fit_is_clean(emdq, polls):
    sc, src, dst = _matches('seq1280', 21)
    clean = emdq.emdq_fit(src, dst, sc.w, sc.h)
    torch.cuda.synchronize()
    ws = clean['workspace']
    bad, ms, wall = _timed(lambda: emdq.emdq_fit(src, dst, sc.w, sc.h, workspace=ws,
                                                 reserved=(polls, 1, 0, 0)))
    info = emdq.read_fit_info(bad['info'])
    print(f'bound {polls or "default"}: ETIMEOUT after {ms:.2f} ms on the device ({wall:.2f} s wall)')
    assert info['status_name'] == 'ETIMEOUT'
    assert wall < (1.0 if polls else 10.0)
    again = emdq.emdq_fit(src, dst, sc.w, sc.h, workspace=ws)
    torch.cuda.synchronize()
    assert emdq.read_fit_info(again['info'])['status_name'] == 'OK'
    for k in ('q', 'c', 'p'):
        assert torch.equal(again[k], clean[k]), k


def test_batched_fits_time_out_together(emdq):
    probs = []
    for seed, name in ((22, 'pair640'), (23, 'seq1280'), (24, 'pair640')):
        sc, src, dst = _matches(name, seed)
        probs.append((src, dst, sc.w, sc.h))
    clean = emdq.emdq_fit_batch(probs)
    torch.cuda.synchronize()
    bad, ms, wall = _timed(lambda: emdq.emdq_fit_batch(probs, reserved=(5000, 1, 0, 0)))
    print(f'3 fits in one launch: ETIMEOUT after {ms:.2f} ms')
    assert wall < 1.0
    for r in bad:
        assert emdq.read_fit_info(r['info'])['status_name'] == 'ETIMEOUT'
    again = emdq.emdq_fit_batch(probs)
    torch.cuda.synchronize()
    for r, c in zip(again, clean):
        assert emdq.read_fit_info(r['info'])['status_name'] == 'OK'
        assert torch.equal(r['q'], c['q']) and torch.equal(r['c'], c['c'])
