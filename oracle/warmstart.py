"""FP64 oracle of the learned EM warm start (test infrastructure only).

The paper has no learned component; this is the reading of the build's warm-start: a
small network predicts each match's initial inlier weight p0 from residuals to its
nearest matches, so that EM starts closer to its answer.  Every step is the plain
definition in float64 numpy; the GPU kernels are checked against it.

Features of match j (16 numbers), from its K = 8 nearest matches k != j by |x_k - x_j|
in the reference frame (ties broken by the lower index; the squared distances are compared
in float32, the kernel's precision, as this is an integer decision):
  - f1_k = log(1 + |(y_k - x_k) - (y_j - x_j)| / 1 px): the residual of neighbour k under
    the translation that match j implies -- a consistency test that needs no fit, so it
    stays informative when many matches are outliers;
  - f2_k = log(1 + |x_k - x_j| / 1 px): the neighbour's distance, the scale against which
    the network weighs the residuals (a smooth field separates nearby matches' motions
    in proportion to their distance);
  - each group of 8 sorted ascending; features = [f1 (8), f2 (8)].
Network: 16 -> 64 (ReLU) -> 64 (ReLU) -> 1 (logistic); loss: mean binary cross-entropy
against the oracle posterior at convergence (soft labels); optimiser: Adam.
Parameter vector (5313 values): W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3[1].
"""
from __future__ import annotations

import numpy as np


K_NN = 8
N_IN, N_H = 16, 64
N_PARAMS = N_H * N_IN + N_H + N_H * N_H + N_H + N_H + 1


def unpack(w):
    w = np.asarray(w, np.float64)
    o = 0
    W1 = w[o:o + N_H * N_IN].reshape(N_H, N_IN); o += N_H * N_IN
    b1 = w[o:o + N_H]; o += N_H
    W2 = w[o:o + N_H * N_H].reshape(N_H, N_H); o += N_H * N_H
    b2 = w[o:o + N_H]; o += N_H
    W3 = w[o:o + N_H]; o += N_H
    b3 = w[o]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), np.atleast_1d(b3)])


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation (the starting point of training)."""
    g = np.random.Generator(np.random.Philox(key=[seed, 77]))
    W1 = g.normal(0, np.sqrt(2.0 / N_IN), (N_H, N_IN))
    W2 = g.normal(0, np.sqrt(2.0 / N_H), (N_H, N_H))
    W3 = g.normal(0, np.sqrt(1.0 / N_H), N_H)
    return pack(W1, np.zeros(N_H), W2, np.zeros(N_H), W3, 0.0)


def knn(src, k: int = K_NN) -> np.ndarray:
    """Indices [n, k] of each match's k nearest other matches (float32 distances)."""
    x = np.asarray(src, np.float32)
    n = x.shape[0]
    out = np.empty((n, k), np.int64)
    for j in range(n):
        dx = (x[:, 0] - x[j, 0]).astype(np.float32)
        dy = (x[:, 1] - x[j, 1]).astype(np.float32)
        d = (dx * dx).astype(np.float32) + (dy * dy).astype(np.float32)
        d = d.astype(np.float32)
        d[j] = np.inf
        order = np.lexsort((np.arange(n), d))      # by distance, then by index
        out[j] = order[:k]
    return out


def features(src, dst) -> np.ndarray:
    """[n, 16] features of every match (see the module docstring)."""
    src = np.asarray(src, np.float64)
    dst = np.asarray(dst, np.float64)
    disp = dst - src
    nn = knn(src)
    n = src.shape[0]
    f = np.empty((n, 2 * K_NN))
    for j in range(n):
        f1 = [np.log1p(np.hypot(*(disp[k] - disp[j]))) for k in nn[j]]
        f2 = [np.log1p(np.hypot(*(src[k] - src[j]))) for k in nn[j]]
        f[j, :K_NN] = np.sort(f1)
        f[j, K_NN:] = np.sort(f2)
    return f


def forward(w, X):
    """Returns (p [B], cache) for features X [B, 16]."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3 + b3
    p = 1.0 / (1.0 + np.exp(-z))
    return p, (X, a1, h1, a2, h2, z, p)


def loss(w, X, y) -> float:
    """Mean binary cross-entropy, written with log-sigmoid for stability."""
    _, (_, _, _, _, _, z, _) = forward(w, X)
    y = np.asarray(y, np.float64)
    # -[y log s(z) + (1-y) log(1 - s(z))] = softplus(z) - y z
    return float(np.mean(np.logaddexp(0.0, z) - y * z))


def grad(w, X, y) -> np.ndarray:
    """Gradient of loss() by the chain rule (backpropagation)."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    p, (X, a1, h1, a2, h2, z, _) = forward(w, X)
    y = np.asarray(y, np.float64)
    B = X.shape[0]
    dz = (p - y) / B                       # d loss / d z
    gW3 = h2.T @ dz
    gb3 = dz.sum()
    dh2 = np.outer(dz, W3) * (a2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(0)
    return pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(w, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma & Ba); t counts from 1.  Returns (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
