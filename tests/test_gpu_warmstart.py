"""GPU parity of the learned EM warm start: features, BF16 inference, gradients and Adam
against the FP64 oracle; training reduces the loss; the shipped network cuts EM
iterations at equal field accuracy."""
import os

import numpy as np
import pytest
import torch

import oracle.warmstart as ows
from synth import make_matches, make_scene, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _pair(seed, n=200, outl=0.25, noise=1.0):
    sc = make_scene(seed, 640, 480, 1)
    s, d, inl = make_matches(sc, 1, n, outl, noise)
    return sc, s, d, inl


def test_features_match_the_oracle(emdq):
    sc, s, d, _ = _pair(31, n=300)
    st, dt = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    got = emdq.warm_features(st, dt).cpu().numpy()
    want = ows.features(np.float32(s).astype(np.float64), np.float32(d).astype(np.float64))
    # same neighbour sets (float32 decisions on both sides); FP32 vs FP64 residuals
    assert np.abs(got - want).max() < 2e-4


def test_batched_warm_start_equals_features_then_network(emdq):
    params = emdq.load_warmstart_params()
    probs = []
    for seed, n in ((41, 200), (42, 1000), (43, 137)):
        sc, s, d, _ = _pair(seed, n=n)
        probs.append((torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()))
    got = emdq.warm_start(probs, params)
    for (st, dt), p in zip(probs, got):
        want = emdq.warm_infer(emdq.warm_features(st, dt), params)
        assert torch.equal(p, want)


def _layout(kind, n, rng):
    """Match positions that stress the grid search: uniform, tight clusters, a line, many
    exact duplicates, a wide empty gap, and a frame with 1 px of height."""
    if kind == 'uniform':
        x = rng.uniform(0, [1920, 1080], (n, 2))
    elif kind == 'clusters':
        c = rng.uniform(0, [1920, 1080], (5, 2))
        x = c[rng.integers(0, 5, n)] + rng.normal(0, 3.0, (n, 2))
    elif kind == 'line':
        x = np.stack([rng.uniform(0, 1920, n), np.full(n, 500.0)], 1)
    elif kind == 'duplicates':
        x = rng.uniform(0, [64, 48], (n, 2)).round()
    elif kind == 'gap':
        x = rng.uniform(0, [100, 100], (n, 2))
        x[: n // 10] += 1800.0
    else:                                                  # 'thin'
        x = np.stack([rng.uniform(0, 1280, n), rng.uniform(0, 1, n)], 1)
    y = x + rng.normal(0, 2.0, (n, 2))
    return x.astype(np.float32), y.astype(np.float32)


@pytest.mark.parametrize('kind', ['uniform', 'clusters', 'line', 'duplicates', 'gap', 'thin'])
def test_batched_warm_start_search_equals_brute_force(emdq, kind):
    """The batched warm start's grid search finds the brute-force neighbours (same p0 bits),
    for n = 9 (the least), ragged sizes, 8192 (the most it stages) and 8193 (past it: the
    batch then takes the brute-force kernel)."""
    params = emdq.load_warmstart_params()
    rng = np.random.default_rng(['uniform', 'clusters', 'line', 'duplicates', 'gap', 'thin'].index(kind))
    for ns in ((9, 10, 300), (1000, 4999), (8192,), (8193, 40)):
        probs = []
        for n in ns:
            x, y = _layout(kind, n, rng)
            probs.append((torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()))
        got = emdq.warm_start(probs, params)
        for (st, dt), p in zip(probs, got):
            want = emdq.warm_infer(emdq.warm_features(st, dt), params)
            assert torch.equal(p, want), (kind, st.shape[0])


def _bf16_forward(w, X):
    """The oracle network with the kernel's BF16 rounding of operands (for the tolerance
    check only; the reference is the FP64 forward)."""
    r = lambda a: torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    W1, b1, W2, b2, W3, b3 = (r(a) for a in ows.unpack(w))
    h1 = r(np.maximum(r(X) @ W1.T + b1, 0))
    h2 = r(np.maximum(h1 @ W2.T + b2, 0))
    return 1 / (1 + np.exp(-(h2 @ W3 + b3)))


def test_inference_matches_the_oracle(emdq):
    g = np.random.default_rng(2)
    w = ows.init_params(5) * 0.7
    X = np.abs(g.normal(0, 1.5, (700, 16)))
    got = emdq.warm_infer(torch.tensor(X, dtype=torch.float32).cuda(),
                          torch.tensor(w, dtype=torch.float32).cuda()).cpu().numpy()
    want, _ = ows.forward(w, np.float32(X).astype(np.float64))
    # BF16 operands (8-bit significands) through three layers
    assert np.abs(got - want).max() < 0.02 and np.abs(got - want).mean() < 0.004
    # against the same rounding emulated in numpy: equal except where an FP32 vs FP64
    # accumulation lands on the other side of a BF16 rounding boundary
    d16 = np.abs(got - _bf16_forward(w, np.float32(X)))
    print('inference vs FP64', np.abs(got - want).max(), 'vs BF16 emulation', np.median(d16), d16.max())
    assert np.median(d16) < 1e-6 and np.percentile(d16, 99) < 2e-3


def test_gradient_and_adam_match_the_oracle(emdq):
    g = np.random.default_rng(3)
    w = ows.init_params(6) * 0.7
    X = np.abs(g.normal(0, 1.5, (1000, 16))).astype(np.float32)
    y = (g.uniform(size=1000) < 0.6).astype(np.float32)
    tw = torch.tensor(w, dtype=torch.float32).cuda()
    grad = torch.zeros_like(tw)
    loss = torch.zeros(1, device='cuda')
    emdq.mlp_train_step(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), tw, None, None, 0,
                        0.0, grad_out=grad, loss_out=loss)
    want_g = ows.grad(w, X.astype(np.float64), y.astype(np.float64))
    got_g = grad.cpu().numpy().astype(np.float64)
    cos = got_g @ want_g / np.linalg.norm(got_g) / np.linalg.norm(want_g)
    print('gradient cosine', cos, 'relative error', np.linalg.norm(got_g - want_g) / np.linalg.norm(want_g))
    assert cos > 0.999 and np.linalg.norm(got_g - want_g) < 0.05 * np.linalg.norm(want_g)
    assert float(loss.item()) == pytest.approx(ows.loss(w, X.astype(np.float64), y), rel=5e-3)
    # one Adam step from zero moments with the kernel's own gradient
    m = torch.zeros_like(tw)
    v = torch.zeros_like(tw)
    tw2 = tw.clone()
    emdq.mlp_train_step(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), tw2, m, v, 1,
                        1e-3, grad_out=grad)
    w_want, m_want, v_want = ows.adam_step(np.float32(w).astype(np.float64),
                                           grad.cpu().numpy().astype(np.float64),
                                           np.zeros_like(w), np.zeros_like(w), 1, 1e-3)
    assert np.abs(tw2.cpu().numpy() - w_want).max() < 1e-6
    # FP32 moments: one rounding of (1 - b1) g
    assert np.all(np.abs(m.cpu().numpy() - m_want) <= 1e-6 * np.abs(m_want) + 1e-12)


def test_training_reduces_the_loss(emdq):
    from warmstart_train import make_training_set
    from paper_2103_07414_gb300.training import train
    feat, label = make_training_set(range(500, 540))
    p0 = torch.from_numpy(ows.init_params(0).astype(np.float32)).cuda()
    l0 = torch.zeros(1, device='cuda')
    emdq.mlp_train_step(feat, label, p0, None, None, 0, 0.0, loss_out=l0)
    params, losses = train(feat, label, steps=400, batch=512, log_every=100)
    l1 = torch.zeros(1, device='cuda')
    emdq.mlp_train_step(feat, label, params, None, None, 0, 0.0, loss_out=l1)
    assert float(l1.item()) < 0.5 * float(l0.item())
    p = emdq.warm_infer(feat, params)
    acc = float(((p >= 0.5) == (label >= 0.5)).float().mean().item())
    assert acc > 0.95


@pytest.mark.skipif(not os.path.exists(os.path.join(os.path.dirname(os.path.dirname(
    os.path.abspath(__file__))), 'paper_2103_07414_gb300', 'warmstart_mlp.npy')),
    reason='no trained warm-start parameters shipped')
def test_shipped_network_cuts_em_iterations(emdq):
    from warmstart_train import evaluate
    params = emdq.load_warmstart_params()
    rows = evaluate(params, seeds=(0, 1, 2))
    it_plain = np.mean([r['plain']['iters'] for r in rows])
    it_warm = np.mean([r['warm']['iters'] for r in rows])
    print('EM iterations plain', it_plain, 'warm', it_warm, rows)
    assert it_warm <= it_plain - 1.0
    for r in rows:
        assert r['warm']['rms'] <= 1.05 * r['plain']['rms'] + 0.02
        assert r['warm']['precision'] >= r['plain']['precision'] - 0.01
        assert r['warm']['recall'] >= r['plain']['recall'] - 0.01
