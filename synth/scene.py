"""Procedural scene, ground-truth deformation, frames, matches and windows.

Coordinates are pixels with the origin at the centre of pixel (0, 0), x to the right and
y down, the convention the paper's warp function uses (Eq. 1: image coordinates in
pixels).  Frame 0 is the reference; frame t is related to it by the ground-truth map

    y = GT_t(x) = s_g (R(theta_g) x + t_g) + sum_b a_b exp(-|x - c_b(t)|^2 / (2 sigma_b^2))

a similarity in the paper's form plus smooth Gaussian displacement bumps whose centres
drift linearly with the frame index.  Frame t's pixel at y shows the texture at
GT_t^{-1}(y), found by Newton's method on the analytic map, and the texture is an
analytic sum of plane waves, so rendering needs no image interpolation.

Random parameters come from numpy's Philox counter-based generator keyed by the seed,
so the same seed gives the same scene on every machine.  Heavy per-pixel evaluation runs
in torch float64 on any device.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch


@dataclass
class Scene:
    w: int
    h: int
    channels: int
    theta: float                 # similarity rotation (rad)
    scale: float                 # similarity scale
    trans: tuple                 # similarity translation (px), inside the scale as in Eq. 1
    bump_c: np.ndarray           # (B, 2) bump centres at frame 0
    bump_a: np.ndarray           # (B, 2) bump displacement vectors (px)
    bump_sigma: float
    bump_drift: np.ndarray       # (B, 2) centre motion per frame (px)
    pan: tuple = (0.0, 0.0)      # extra translation per frame (px, frame coordinates)
    pan_turn: int = 0            # > 0: the pan reverses every pan_turn frames (out and back,
                                 # so the camera is over the start again at frame 2 pan_turn)
    wave_k: np.ndarray = field(default=None)     # (K, 2) wave vectors (rad/px)
    wave_phi: np.ndarray = field(default=None)   # (K,) phases
    wave_amp: np.ndarray = field(default=None)   # (C, K) per-channel amplitudes
    seed: int = 0


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & 0xFFFFFFFFFFFFFFFF, stream]))


def make_scene(seed: int, w: int, h: int, channels: int = 3, rot_deg: float = 5.0,
               scale: float = 1.05, trans=(12.0, -7.0), n_bumps: int = 3,
               bump_amp: float = 8.0, bump_sigma: float = 60.0, drift: float = 0.0,
               pan=(0.0, 0.0), pan_turn: int = 0) -> Scene:
    """Draw a scene: texture waves, bump centres/directions and drift directions."""
    g = _rng(seed, 1)
    bump_c = np.stack([g.uniform(0.15 * w, 0.85 * w, n_bumps),
                       g.uniform(0.15 * h, 0.85 * h, n_bumps)], axis=1)
    ang = g.uniform(0.0, 2.0 * math.pi, n_bumps)
    bump_a = bump_amp * np.stack([np.cos(ang), np.sin(ang)], axis=1)
    dang = g.uniform(0.0, 2.0 * math.pi, n_bumps)
    bump_drift = drift * np.stack([np.cos(dang), np.sin(dang)], axis=1)
    # texture: 4 octaves x 8 plane waves, amplitude growing with wavelength (smooth noise)
    lam = []
    for base in (96.0, 48.0, 24.0, 12.0):
        lam.append(base * g.uniform(0.75, 1.25, 8))
    lam = np.concatenate(lam)
    dirs = g.uniform(0.0, 2.0 * math.pi, lam.size)
    wave_k = (2.0 * math.pi / lam)[:, None] * np.stack([np.cos(dirs), np.sin(dirs)], axis=1)
    wave_phi = g.uniform(0.0, 2.0 * math.pi, lam.size)
    amp = lam ** 0.8
    amp = amp / math.sqrt(0.5 * float(np.sum(amp ** 2))) * 45.0   # ~45 grey levels std
    wave_amp = np.stack([amp * g.uniform(0.6, 1.0, lam.size) for _ in range(channels)])
    return Scene(w=w, h=h, channels=channels, theta=math.radians(rot_deg), scale=scale,
                 trans=tuple(float(v) for v in trans), bump_c=bump_c, bump_a=bump_a,
                 bump_sigma=float(bump_sigma), bump_drift=bump_drift,
                 pan=tuple(float(v) for v in pan), pan_turn=int(pan_turn), wave_k=wave_k,
                 wave_phi=wave_phi,
                 wave_amp=wave_amp, seed=seed)


def _t(a, like: torch.Tensor) -> torch.Tensor:
    return torch.as_tensor(np.asarray(a), dtype=torch.float64, device=like.device)


def pan_frames(sc: Scene, t: int) -> float:
    """Frames of pan travel at frame t: t, or a triangle wave of period 2 pan_turn."""
    if sc.pan_turn <= 0:
        return float(t)
    ph = int(t) % (2 * sc.pan_turn)
    return float(ph if ph <= sc.pan_turn else 2 * sc.pan_turn - ph)


def _similarity_shift(sc: Scene, t: int):
    k = pan_frames(sc, t)
    return sc.trans[0] + sc.pan[0] * k / sc.scale, sc.trans[1] + sc.pan[1] * k / sc.scale


def gt_forward(sc: Scene, x: torch.Tensor, t: int) -> torch.Tensor:
    """Ground-truth map from reference coordinates x[..., 2] to frame-t coordinates."""
    x = x.to(torch.float64)
    c, s = math.cos(sc.theta), math.sin(sc.theta)
    tx, ty = _similarity_shift(sc, t)
    y0 = sc.scale * (c * x[..., 0] - s * x[..., 1] + tx)
    y1 = sc.scale * (s * x[..., 0] + c * x[..., 1] + ty)
    cen = _t(sc.bump_c + t * sc.bump_drift, x)
    amp = _t(sc.bump_a, x)
    d = x[..., None, :] - cen                                  # [..., B, 2]
    gb = torch.exp(-(d * d).sum(-1) / (2.0 * sc.bump_sigma ** 2))  # [..., B]
    y0 = y0 + (gb * amp[:, 0]).sum(-1)
    y1 = y1 + (gb * amp[:, 1]).sum(-1)
    return torch.stack([y0, y1], dim=-1)


def _gt_jacobian(sc: Scene, x: torch.Tensor, t: int) -> torch.Tensor:
    c, s = math.cos(sc.theta), math.sin(sc.theta)
    J = torch.empty(x.shape[:-1] + (2, 2), dtype=torch.float64, device=x.device)
    J[..., 0, 0] = sc.scale * c
    J[..., 0, 1] = -sc.scale * s
    J[..., 1, 0] = sc.scale * s
    J[..., 1, 1] = sc.scale * c
    cen = _t(sc.bump_c + t * sc.bump_drift, x)
    amp = _t(sc.bump_a, x)
    d = x[..., None, :] - cen
    gb = torch.exp(-(d * d).sum(-1) / (2.0 * sc.bump_sigma ** 2))
    grad = -(gb[..., None] * d) / sc.bump_sigma ** 2           # [..., B, 2]
    J = J + torch.einsum('bi,...bj->...ij', amp, grad)
    return J


def gt_inverse(sc: Scene, y: torch.Tensor, t: int, iters: int = 10) -> torch.Tensor:
    """Invert the ground-truth map by Newton's method (generator-only)."""
    y = y.to(torch.float64)
    c, s = math.cos(sc.theta), math.sin(sc.theta)
    tx, ty = _similarity_shift(sc, t)
    u0 = y[..., 0] / sc.scale - tx
    u1 = y[..., 1] / sc.scale - ty
    x = torch.stack([c * u0 + s * u1, -s * u0 + c * u1], dim=-1)   # similarity inverse
    for _ in range(iters):
        r = gt_forward(sc, x, t) - y
        J = _gt_jacobian(sc, x, t)
        det = J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
        dx0 = (J[..., 1, 1] * r[..., 0] - J[..., 0, 1] * r[..., 1]) / det
        dx1 = (-J[..., 1, 0] * r[..., 0] + J[..., 0, 0] * r[..., 1]) / det
        x = x - torch.stack([dx0, dx1], dim=-1)
    return x


def texture(sc: Scene, x: torch.Tensor) -> torch.Tensor:
    """Analytic texture value at reference coordinates x[..., 2] -> [..., C] in [0, 255]."""
    x = x.to(torch.float64)
    k = _t(sc.wave_k, x)
    ph = _t(sc.wave_phi, x)
    amp = _t(sc.wave_amp, x)                                   # [C, K]
    out = []
    flat = x.reshape(-1, 2)
    for ch in range(sc.channels):
        acc = torch.full(flat.shape[:1], 128.0, dtype=torch.float64, device=x.device)
        # chunk over waves to bound memory at large frames
        for k0 in range(0, k.shape[0], 8):
            arg = flat @ k[k0:k0 + 8].T + ph[k0:k0 + 8]
            acc = acc + (torch.cos(arg) * amp[ch, k0:k0 + 8]).sum(-1)
        out.append(acc)
    v = torch.stack(out, dim=-1).clamp_(0.0, 255.0)
    return v.reshape(x.shape[:-1] + (sc.channels,))


def _pixel_grid(w: int, h: int, device) -> torch.Tensor:
    ys, xs = torch.meshgrid(torch.arange(h, dtype=torch.float64, device=device),
                            torch.arange(w, dtype=torch.float64, device=device), indexing='ij')
    return torch.stack([xs, ys], dim=-1)


def _quantise(v: torch.Tensor) -> torch.Tensor:
    return torch.floor(v + 0.5).clamp_(0, 255).to(torch.uint8)


def render_reference(sc: Scene, device='cpu') -> torch.Tensor:
    """Frame 0: the texture at integer reference pixels, uint8 [h, w, C]."""
    return _quantise(texture(sc, _pixel_grid(sc.w, sc.h, device)))


def render_frame(sc: Scene, t: int, device='cpu', rows_per_chunk: int = 256) -> torch.Tensor:
    """Frame t: pixel y shows the texture at GT_t^{-1}(y); uint8 [h, w, C]."""
    out = torch.empty((sc.h, sc.w, sc.channels), dtype=torch.uint8, device=device)
    for r0 in range(0, sc.h, rows_per_chunk):
        r1 = min(sc.h, r0 + rows_per_chunk)
        ys, xs = torch.meshgrid(torch.arange(r0, r1, dtype=torch.float64, device=device),
                                torch.arange(sc.w, dtype=torch.float64, device=device),
                                indexing='ij')
        y = torch.stack([xs, ys], dim=-1)
        out[r0:r1] = _quantise(texture(sc, gt_inverse(sc, y, t)))
    return out


def make_matches(sc: Scene, t: int, n: int, outlier_frac: float, noise_sigma: float,
                 seed: int | None = None):
    """Feature matches between the reference and frame t.

    Returns (src [n,2] float32, dst [n,2] float32, inlier bool[n]) as numpy arrays.
    Inliers: src uniform over the reference, dst = GT_t(src) + N(0, noise^2 I), kept only
    when dst lies inside frame t (a feature must be visible in both frames).  Outliers:
    src and dst independent and uniform over their frames.  Inlier/outlier order is
    shuffled.
    """
    g = _rng(sc.seed if seed is None else seed, 1000 + int(t))
    n_out = int(round(outlier_frac * n))
    n_in = n - n_out
    src_in = np.empty((0, 2))
    dst_in = np.empty((0, 2))
    while src_in.shape[0] < n_in:
        m = 2 * (n_in - src_in.shape[0]) + 16
        x = np.stack([g.uniform(0, sc.w - 1, m), g.uniform(0, sc.h - 1, m)], axis=1)
        y = gt_forward(sc, torch.from_numpy(x), t).numpy()
        y = y + g.normal(0.0, noise_sigma, y.shape)
        ok = (y[:, 0] >= 0) & (y[:, 0] <= sc.w - 1) & (y[:, 1] >= 0) & (y[:, 1] <= sc.h - 1)
        src_in = np.concatenate([src_in, x[ok]])[:n_in]
        dst_in = np.concatenate([dst_in, y[ok]])[:n_in]
    src_out = np.stack([g.uniform(0, sc.w - 1, n_out), g.uniform(0, sc.h - 1, n_out)], axis=1)
    dst_out = np.stack([g.uniform(0, sc.w - 1, n_out), g.uniform(0, sc.h - 1, n_out)], axis=1)
    src = np.concatenate([src_in, src_out])
    dst = np.concatenate([dst_in, dst_out])
    inl = np.concatenate([np.ones(n_in, bool), np.zeros(n_out, bool)])
    perm = g.permutation(n)
    return (src[perm].astype(np.float32), dst[perm].astype(np.float32), inl[perm])


def make_pair_matches(sc: Scene, t0: int, t1: int, n: int, outlier_frac: float,
                      noise_sigma: float, seed: int | None = None):
    """Feature matches between frames t0 and t1 (frame 0 is the reference itself).

    A feature is a reference point x seen at x in frame 0 and at GT_t(x) in frame t >= 1;
    inliers: x uniform over the reference, src = its position in frame t0, dst = its position in
    frame t1 plus N(0, noise^2 I), kept when both lie inside their frames; outliers: src and dst
    independent and uniform over the frame.  Returns (src, dst [n, 2] float32, inlier bool[n],
    x [n, 2] float64: the inliers' reference points, NaN for outliers)."""
    g = _rng(sc.seed if seed is None else seed, 5000 + 97 * int(t0) + int(t1))
    n_out = int(round(outlier_frac * n))
    n_in = n - n_out

    def at(t, x):
        return x if t == 0 else gt_forward(sc, torch.from_numpy(x), t).numpy()

    xs, a, b = np.empty((0, 2)), np.empty((0, 2)), np.empty((0, 2))
    while xs.shape[0] < n_in:
        m = 2 * (n_in - xs.shape[0]) + 16
        x = np.stack([g.uniform(0, sc.w - 1, m), g.uniform(0, sc.h - 1, m)], axis=1)
        p0 = at(t0, x)
        p1 = at(t1, x) + g.normal(0.0, noise_sigma, x.shape)
        ok = ((p0[:, 0] >= 0) & (p0[:, 0] <= sc.w - 1) & (p0[:, 1] >= 0) & (p0[:, 1] <= sc.h - 1) &
              (p1[:, 0] >= 0) & (p1[:, 0] <= sc.w - 1) & (p1[:, 1] >= 0) & (p1[:, 1] <= sc.h - 1))
        xs = np.concatenate([xs, x[ok]])[:n_in]
        a = np.concatenate([a, p0[ok]])[:n_in]
        b = np.concatenate([b, p1[ok]])[:n_in]
    oa = np.stack([g.uniform(0, sc.w - 1, n_out), g.uniform(0, sc.h - 1, n_out)], axis=1)
    ob = np.stack([g.uniform(0, sc.w - 1, n_out), g.uniform(0, sc.h - 1, n_out)], axis=1)
    src = np.concatenate([a, oa])
    dst = np.concatenate([b, ob])
    inl = np.concatenate([np.ones(n_in, bool), np.zeros(n_out, bool)])
    xr = np.concatenate([xs, np.full((n_out, 2), np.nan)])
    perm = g.permutation(n)
    return src[perm].astype(np.float32), dst[perm].astype(np.float32), inl[perm], xr[perm]


def canvas_origin(canvas_w: int, canvas_h: int, w0: int, h0: int):
    """Canvas position of reference pixel (0, 0): the reference frame is centred."""
    return ((canvas_w - w0) // 2, (canvas_h - h0) // 2)


def footprint_window(sc: Scene, t: int, canvas_w: int, canvas_h: int, pad: int = 2):
    """Bounding box, in reference coordinates, of frame t's footprint under GT_t^{-1}.

    Expanded by `pad` pixels and clipped to the canvas.  Returns (x0, y0, gw, gh).
    """
    w, h = sc.w, sc.h
    e = []
    xs = np.arange(0, w, 4.0)
    ys = np.arange(0, h, 4.0)
    for yy in (0.0, h - 1.0):
        e.append(np.stack([xs, np.full_like(xs, yy)], 1))
    for xx in (0.0, w - 1.0):
        e.append(np.stack([np.full_like(ys, xx), ys], 1))
    e.append(np.array([[w - 1.0, h - 1.0]]))
    b = gt_inverse(sc, torch.from_numpy(np.concatenate(e)), t).numpy()
    ox, oy = canvas_origin(canvas_w, canvas_h, w, h)
    x0 = max(int(math.floor(b[:, 0].min())) - pad, -ox)
    y0 = max(int(math.floor(b[:, 1].min())) - pad, -oy)
    x1 = min(int(math.ceil(b[:, 0].max())) + pad, canvas_w - 1 - ox)
    y1 = min(int(math.ceil(b[:, 1].max())) + pad, canvas_h - 1 - oy)
    return (x0, y0, max(0, x1 - x0 + 1), max(0, y1 - y0 + 1))


# The workloads: sizes, match counts and outlier rates of the paper's laparoscopy
# sequences scaled to current video formats.
WORKLOADS = {
    # one pair, 640x480 grey, N=200, 20% outliers, noise 1 px, canvas 1024^2
    'pair640': dict(w=640, h=480, channels=1, n=200, outliers=0.2, noise=1.0,
                    canvas=(1024, 1024), drift=0.0, frames=1),
    # 100-frame sequence, 1280x1024 RGB, N=1000, 30% outliers, noise 1.5 px,
    # bumps drifting 2 px/frame, canvas 4096^2
    'seq1280': dict(w=1280, h=1024, channels=3, n=1000, outliers=0.3, noise=1.5,
                    canvas=(4096, 4096), drift=2.0, frames=100),
    # learned warm-start evaluation: 1280x1024, N=2000, 40% outliers
    'warm2000': dict(w=1280, h=1024, channels=3, n=2000, outliers=0.4, noise=1.5,
                     canvas=(4096, 4096), drift=0.0, frames=1),
    # full sequence: 500 frames 1920x1080 RGB, N=5000, 30% outliers, bumps drifting 1 px/frame,
    # camera pan of 6 px/frame (at 30 degrees to the x axis) out for 200 frames and back, so
    # frame 400 revisits the start; fits batched 8 frames per launch; canvas 8192^2
    'seq1920': dict(w=1920, h=1080, channels=3, n=5000, outliers=0.3, noise=1.5,
                    canvas=(8192, 8192), drift=1.0, frames=500,
                    pan=(6.0 * math.cos(math.radians(30.0)), 6.0 * math.sin(math.radians(30.0))),
                    pan_turn=200, batch=8),
}


def workload(name: str, seed: int = 0) -> tuple[Scene, dict]:
    cfg = dict(WORKLOADS[name])
    sc = make_scene(seed, cfg['w'], cfg['h'], cfg['channels'], drift=cfg['drift'],
                    pan=cfg.get('pan', (0.0, 0.0)), pan_turn=cfg.get('pan_turn', 0))
    return sc, cfg


# Mixed-size batch: independent frame pairs of uneven sizes and match counts.
MIXED_SIZES = ((640, 480), (1280, 720), (1280, 1024), (1920, 1080))


def mixed_pairs(seed: int, count: int = 64, channels: int = 3, n_range=(100, 3000),
                outlier_range=(0.10, 0.40), noise: float = 1.0):
    """`count` independent pairs: frame size uniform over MIXED_SIZES, N uniform in
    n_range (inclusive), outlier rate uniform in outlier_range; each pair its own scene
    (reference frame and frame 1).  Returns a list of dicts (scene, src, dst, inlier, n,
    outliers)."""
    g = _rng(seed, 5)
    pairs = []
    for b in range(count):
        w, h = MIXED_SIZES[int(g.integers(0, len(MIXED_SIZES)))]
        n = int(g.integers(n_range[0], n_range[1] + 1))
        outl = float(g.uniform(*outlier_range))
        sc = make_scene(seed * 1000 + b, w, h, channels)
        s, d, inl = make_matches(sc, 1, n, outl, noise)
        pairs.append(dict(scene=sc, src=s, dst=d, inlier=inl, n=n, outliers=outl))
    return pairs
