"""GPU parity: emdq_fit_batch runs several fits of different sizes in one launch; each
must agree with its own emdq_fit and with the oracle."""
import numpy as np
import pytest
import torch

from synth import make_matches, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _apply(q8, x):
    a, b, u, v, s = (q8[:, k] for k in range(5))
    n2 = a * a + b * b
    X = ((a * a - b * b) * x[:, 0] - 2 * a * b * x[:, 1] + 2 * (a * u - b * v)) / n2
    Y = (2 * a * b * x[:, 0] + (a * a - b * b) * x[:, 1] + 2 * (b * u + a * v)) / n2
    return s[:, None] * np.stack([X, Y], 1)


def test_batch_matches_single_fits_and_oracle(emdq, orc):
    cases = []
    for name, seed, t in [('pair640', 1, 1), ('seq1280', 2, 10), ('seq1280', 2, 11), ('warm2000', 3, 1),
                          ('pair640', 4, 1)]:
        sc, cfg = workload(name, seed=seed)
        s, d, _ = make_matches(sc, t, cfg['n'], cfg['outliers'], cfg['noise'])
        cases.append((sc, s, d))
    probs = [(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), sc.w, sc.h) for sc, s, d in cases]
    res = emdq.emdq_fit_batch(probs)
    torch.cuda.synchronize()
    for (sc, s, d), pr, r in zip(cases, probs, res):
        info = emdq.read_fit_info(r['info'])
        single = emdq.emdq_fit(*pr)
        sinfo = emdq.read_fit_info(single['info'])
        assert info['status_name'] == sinfo['status_name'] == 'OK'
        assert info['iters'] == sinfo['iters']
        # converged EM results are defined up to the stopping tolerance (max |dp| < 1e-3):
        # other CTA groupings sum the sigma^2 partials in another FP32 order
        assert (r['p'] - single['p']).abs().max().item() <= 1e-3
        f64 = lambda a: np.float32(a).astype(np.float64)
        want = orc.fit(f64(s), f64(d), sc.w, sc.h)
        assert info['iters'] == want['iters']
        got_p = r['p'].cpu().numpy()
        assert np.abs(got_p - want['p']).max() <= 1e-3
        sure = np.abs(want['p'] - 0.5) > 0.1
        np.testing.assert_array_equal((r['c'].cpu().numpy() > 0)[sure], (want['c'] > 0)[sure])
        dpos = np.abs(_apply(r['q'].cpu().numpy().astype(np.float64), f64(s)) -
                      _apply(want['q8'], f64(s)))[want['c'] > 0].max()
        assert dpos <= 2e-3


def test_batch_argument_errors(emdq):
    x = torch.zeros((10, 2), device='cuda')
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_fit_batch([(x[:2], x[:2], 640, 480)])
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_fit_batch([(x, x, 640, 480)] * 65)


def _mixed_problems(seed, count):
    """(scene, src, dst) of the mixed-size batch recipe."""
    from synth import mixed_pairs
    return [(p['scene'], p['src'], p['dst']) for p in mixed_pairs(seed, count)]


def test_mixed_batch_split_does_not_change_results(emdq):
    """The CTA split (default n^2 policy, uniform, autotuned) changes only the FP32 order of
    the sigma^2 partial sums: every split gives each problem its own emdq_fit result to the
    stopping tolerance."""
    cases = _mixed_problems(7, 12)
    probs = [(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), sc.w, sc.h) for sc, s, d in cases]
    cap = emdq.fit_batch_capacity(probs)
    assert cap >= len(probs)
    useful = [(p[0].shape[0] + 7) // 8 for p in probs]
    uniform = [min(u, cap // len(probs)) for u in useful]
    tuned, ms = emdq.fit_batch_autotune(probs, reps=1)
    assert ms > 0 and sum(tuned) <= cap and all(1 <= t <= u for t, u in zip(tuned, useful))
    runs = [emdq.emdq_fit_batch(probs), emdq.emdq_fit_batch(probs, ctas=uniform),
            emdq.emdq_fit_batch(probs, ctas=tuned)]
    torch.cuda.synchronize()
    for b, pr in enumerate(probs):
        single = emdq.emdq_fit(*pr)
        for r in runs:
            assert emdq.read_fit_info(r[b]['info'])['status_name'] == 'OK'
            assert (r[b]['p'] - single['p']).abs().max().item() <= 1e-3
            assert torch.equal(r[b]['c'] > 0, single['c'] > 0) or \
                ((r[b]['c'] > 0) != (single['c'] > 0)).sum().item() <= 1


def test_mixed_batch_of_64(emdq, orc):
    """64 mixed pairs in one launch; a sample of them against the oracle."""
    cases = _mixed_problems(11, 64)
    probs = [(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), sc.w, sc.h) for sc, s, d in cases]
    res = emdq.emdq_fit_batch(probs)
    torch.cuda.synchronize()
    f64 = lambda a: np.float32(a).astype(np.float64)
    for b in (0, 17, 40, 63):
        sc, s, d = cases[b]
        info = emdq.read_fit_info(res[b]['info'])
        want = orc.fit(f64(s), f64(d), sc.w, sc.h)
        assert info['status_name'] == 'OK'
        assert abs(info['iters'] - want['iters']) <= 1
        assert np.abs(res[b]['p'].cpu().numpy() - want['p']).max() <= 2e-3


def test_batch_split_errors(emdq):
    x = torch.rand((40, 2), device='cuda') * 100
    probs = [(x, x + 1, 640, 480)] * 3
    cap = emdq.fit_batch_capacity(probs)
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_fit_batch(probs, ctas=[0, 1, 1])
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_fit_batch(probs, ctas=[cap, 1, 1])
    with pytest.raises(ValueError):
        emdq.emdq_fit_batch(probs, ctas=[1, 1])
