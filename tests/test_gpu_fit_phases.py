"""GPU parity of emdq_fit_batch_phases: a batch fitted in phases (the unconverged fits continued,
with every CTA, from their posteriors) runs the same EM iteration as one launch.

  - fixed rounds (tol 0) split over three phases against the oracle's FP64 fit with as many
    rounds, by the criteria of the single-fit parity test;
  - a mixed batch: fits that end in the first phase are bit for bit those of one launch, the
    continued ones agree with it (status, iterations within one, inlier decisions, rows);
  - one phase is the plain batch launch, bit for bit.
"""
import numpy as np
import pytest
import torch

from synth import make_matches, mixed_pairs, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _apply(q8, x):
    """Warp of each row applied to its own match position (the row's prediction)."""
    a, b, u, v, s = (q8[:, k] for k in range(5))
    n2 = a * a + b * b
    X = ((a * a - b * b) * x[:, 0] - 2 * a * b * x[:, 1] + 2 * (a * u - b * v)) / n2
    Y = (2 * a * b * x[:, 0] + (a * a - b * b) * x[:, 1] + 2 * (b * u + a * v)) / n2
    return s[:, None] * np.stack([X, Y], 1)


def _np(r):
    return {k: r[k].cpu().numpy() for k in ('q', 'c', 'p', 'info')}


def test_fixed_rounds_in_three_phases_against_the_oracle(emdq, orc):
    """tol 0: every fit runs 2, then 1, then 2 rounds (ENOCONV after each phase, 5 in all)."""
    cases = []
    for name, seed in (('pair640', 4), ('seq1280', 4), ('seq1280', 5)):
        sc, cfg = workload(name, seed=seed)
        src, dst, _ = make_matches(sc, 1, cfg['n'], cfg['outliers'], cfg['noise'])
        cases.append((sc, src, dst))
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    probs = [(t(src), t(dst), sc.w, sc.h) for sc, src, dst in cases]
    got = emdq.emdq_fit_batch(probs, tol_p=0.0, phases=[2, 3, 5])
    torch.cuda.synchronize()
    for (sc, src, dst), g in zip(cases, got):
        info = emdq.read_fit_info(g['info'])
        assert info['status_name'] == 'ENOCONV' and info['iters'] == 5, info
        want = orc.fit(_f32(src), _f32(dst), sc.w, sc.h, max_iters=5, tol_p=0.0)
        q8 = g['q'].cpu().numpy().astype(np.float64)
        p = g['p'].cpu().numpy().astype(np.float64)
        dp = np.abs(p - want['p']).max()
        dpos = np.abs(_apply(q8, _f32(src)) - _apply(want['q8'], _f32(src))).max()
        print(f'{sc.w}x{sc.h}: max |dp| {dp:.2e}, row diff {dpos:.2e} px, sigma2 {info["sigma2"]:.6f} '
              f'vs {want["sigma2"]:.6f}')
        assert dp <= 1e-4
        assert dpos <= 2e-3
        assert info['sigma2'] == pytest.approx(want['sigma2'], rel=1e-5)
        assert info['gamma'] == pytest.approx(want['gamma'], abs=1e-5)
        np.testing.assert_array_equal(q8[:, 5:], np.tile([1, 0, 0], (len(src), 1)))


def _mixed_problems(emdq, count):
    dev = 'cuda'
    pairs = mixed_pairs(7, count, n_range=(100, 3000))
    src = [torch.from_numpy(p['src']).to(dev) for p in pairs]
    dst = [torch.from_numpy(p['dst']).to(dev) for p in pairs]
    p0 = emdq.warm_start(list(zip(src, dst)), emdq.load_warmstart_params(dev))
    return [(s, d, p['scene'].w, p['scene'].h, q) for s, d, p, q in zip(src, dst, pairs, p0)]


def test_mixed_batch_in_phases_against_one_launch(emdq):
    probs = _mixed_problems(emdq, 24)
    one = [_np(r) for r in emdq.emdq_fit_batch(probs)]
    ph = [_np(r) for r in emdq.emdq_fit_batch(probs, phases=[6, 10, 14, 20])]
    torch.cuda.synchronize()
    cont = 0
    for b, (a, g) in enumerate(zip(one, ph)):
        ia, ig = a['info'], g['info']
        if ia[1] <= 6:
            # ended within the first phase: the same launch arithmetic
            for k in ('q', 'c', 'p', 'info'):
                np.testing.assert_array_equal(a[k], g[k], err_msg=f'{b} {k}')
            continue
        cont += 1
        assert ig[0] == ia[0], (b, ia, ig)                      # status
        assert abs(int(ig[1]) - int(ia[1])) <= 1, (b, ia, ig)   # rounds, within one
        sure = np.abs(a['p'] - 0.5) > 0.1
        np.testing.assert_array_equal((g['c'] > 0)[sure], (a['c'] > 0)[sure])
        x = probs[b][0].cpu().numpy().astype(np.float64)
        inl = a['c'] > 0
        dpos = np.abs(_apply(g['q'].astype(np.float64), x) - _apply(a['q'].astype(np.float64), x))[inl].max()
        assert dpos <= 2e-3, (b, dpos)
    print(f'{cont} of {len(probs)} fits continued past the first phase')
    assert cont > 0


def test_one_phase_is_the_batch_launch(emdq):
    probs = _mixed_problems(emdq, 8)
    one = [_np(r) for r in emdq.emdq_fit_batch(probs, max_iters=20)]
    ph = [_np(r) for r in emdq.emdq_fit_batch(probs, phases=[20])]
    torch.cuda.synchronize()
    for a, g in zip(one, ph):
        for k in ('q', 'c', 'p', 'info'):
            np.testing.assert_array_equal(a[k], g[k])
