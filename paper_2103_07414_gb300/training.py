"""Training of the learned EM warm start on the GPU, in the library's own kernels.

The network (16 -> 64 -> 64 -> 1, ReLU, logistic output; parameters packed as W1[64][16],
b1[64], W2[64][64], b2[64], W3[64], b3) predicts each match's starting inlier weight p0 from
the 16 nearest-neighbour features of ``warm_features``.  ``train`` runs Adam on the mean binary
cross-entropy against given labels (soft labels in [0, 1]: the converged EM posterior of the
same matches), one ``mlp_train_step`` launch per mini-batch, with a cosine-decayed learning
rate.  The labels are the caller's: they come from a reference EMDQ fit of the training
matches, which is not part of this package.
"""
from __future__ import annotations

import math

import torch

N_IN, N_H = 16, 64


def init_params(seed: int = 0, device='cuda') -> torch.Tensor:
    """He-normal weights (variance 2 / fan-in for the ReLU layers, 1 / fan-in for the output
    layer) and zero biases, in the packed layout the kernels read."""
    g = torch.Generator(device='cpu')
    g.manual_seed(int(seed))
    W1 = torch.randn((N_H, N_IN), generator=g, dtype=torch.float64) * math.sqrt(2.0 / N_IN)
    W2 = torch.randn((N_H, N_H), generator=g, dtype=torch.float64) * math.sqrt(2.0 / N_H)
    W3 = torch.randn(N_H, generator=g, dtype=torch.float64) * math.sqrt(1.0 / N_H)
    z = torch.zeros(N_H, dtype=torch.float64)
    p = torch.cat([W1.reshape(-1), z, W2.reshape(-1), z, W3, torch.zeros(1, dtype=torch.float64)])
    return p.to(torch.float32).to(device)


def train(feat: torch.Tensor, label: torch.Tensor, steps: int = 3000, batch: int = 1024,
          lr: float = 3e-3, seed: int = 0, log_every: int = 0, params: torch.Tensor | None = None):
    """Adam on the mean cross-entropy of (feat [M, 16], label [M]) on the device: mini-batches
    drawn without replacement (a new permutation each epoch), learning rate
    lr (1 + cos(pi (step - 1) / steps)) / 2.  Returns (params, [(step, loss), ...])."""
    from . import lib, mlp_train_step
    dev = feat.device
    if params is None:
        params = init_params(seed, dev)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    loss = torch.zeros(1, device=dev)
    xb = torch.empty((batch, N_IN), device=dev)
    yb = torch.empty(batch, device=dev)
    ws = torch.empty(lib().emdq_mlp_train_workspace_size(batch), dtype=torch.uint8, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    M = feat.shape[0]
    perm = torch.randperm(M, device=dev, generator=gen)
    pos = 0
    losses = []
    for step in range(1, steps + 1):
        if pos + batch > M:
            perm = torch.randperm(M, device=dev, generator=gen)
            pos = 0
        idx = perm[pos:pos + batch]
        pos += batch
        torch.index_select(feat, 0, idx, out=xb)
        torch.index_select(label, 0, idx, out=yb)
        lr_t = 0.5 * lr * (1.0 + math.cos(math.pi * (step - 1) / steps))
        mlp_train_step(xb, yb, params, m, v, step, lr_t, loss_out=loss, workspace=ws)
        if log_every and step % log_every == 0:
            losses.append((step, float(loss.item())))
    return params, losses
