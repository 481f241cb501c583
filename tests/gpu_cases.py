"""Seeded cases shared by the GPU parity tests (inputs only; expected values come from
the oracle)."""
import math

import numpy as np

from synth import make_matches, workload


def fitted_case(orc, name='pair640', seed=0, t=1):
    """Matches of a workload and the oracle's fit of them (q rows, weights)."""
    sc, cfg = workload(name, seed=seed)
    src, dst, inl = make_matches(sc, t, cfg['n'], cfg['outliers'], cfg['noise'])
    r = orc.fit(src, dst, sc.w, sc.h)
    return sc, cfg, src, dst, inl, r


def random_rows(rng, n, w, h):
    """n plausible warp rows (similarities near one global motion) and positions."""
    src = np.stack([rng.uniform(0, w - 1, n), rng.uniform(0, h - 1, n)], 1)
    q8 = np.zeros((n, 8))
    th = math.radians(5) + rng.normal(0, 0.01, n)
    s = 1.05 + rng.normal(0, 0.01, n)
    tx = 12 + rng.normal(0, 3, n)
    ty = -7 + rng.normal(0, 3, n)
    c, sn = np.cos(th / 2), np.sin(th / 2)
    q8[:, 0], q8[:, 1] = c, sn
    q8[:, 2] = 0.5 * (tx * c + ty * sn)
    q8[:, 3] = 0.5 * (ty * c - tx * sn)
    q8[:, 4], q8[:, 5] = s, 1.0
    return src, q8
