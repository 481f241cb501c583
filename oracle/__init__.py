"""FP64 CPU oracle of the EMDQ field + mosaic path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product library never does; it and this oracle share no code.
The arithmetic lives in ``emdq_oracle.c`` (plain C, double precision, optional OpenMP
over pixels as the paper's CPU path uses); this module only builds and marshals.

Parity status: every routine here is pinned by ``tests/test_oracle_*.py`` against closed
forms, an independent 8-D dual-quaternion implementation, an SVD solution of the rotation
fit, brute force on tiny inputs and statistical recovery of a known field.  The EM loop
as a whole follows a reading of an algorithm the paper delegates to its EMDQ reference;
its invariants are pinned, its agreement with that reference is not (parity unpinned
against the original EMDQ).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, 'emdq_oracle.c')
_LIB_PATH = os.path.join(_HERE, 'liboracle.so')
_lock = threading.Lock()
_lib = None

OK, EINVAL, EDEGENERATE, ENOCONV = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile emdq_oracle.c into liboracle.so (OpenMP when the compiler has it)."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(os.path.join(_HERE, 'emdq_oracle.h'))):
        return _LIB_PATH
    base = ['gcc', '-O2', '-std=c11', '-fPIC', '-shared', '-ffp-contract=off',
            '-fno-fast-math', _SRC, '-o', _LIB_PATH + '.tmp', '-lm']
    try:
        subprocess.run(base[:1] + ['-fopenmp'] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + '.tmp', _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [('alpha', ctypes.c_double), ('max_iters', ctypes.c_int),
                ('tol_p', ctypes.c_double), ('sigma2_floor', ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            D, I = ctypes.c_double, ctypes.c_int
            L.orc_alpha_for_frame.restype = D
            L.orc_alpha_for_frame.argtypes = [I, I]
            L.orc_beta_for_frame.restype = D
            L.orc_beta_for_frame.argtypes = [I, I]
            L.orc_uncertainty.argtypes = [P, P, I, I, I, I, I, D, P, I]
            L.orc_compose.argtypes = [P, P, P]
            L.orc_node_track.argtypes = [P, P, P, I, P, P, P, I, D, D, P, P, I]
            L.orc_node_merge.argtypes = [P, P, P, P, P, P, I, D, P, P]
            L.orc_arap_smooth.argtypes = [P, P, P, I, D, I, P, P]
            L.orc_arap_fit.argtypes = [P, P, I, D, P, P, P, P]
            L.orc_node_restrict.argtypes = [P, P, I, P, P, I, D, P]
            L.orc_node_init.argtypes = [P, P, I, P, I, D, P]
            L.orc_feature_uncertainty.argtypes = [P, P, I, P, P, D, D, P, P]
            L.orc_keyframe_distances.argtypes = [P, P, I, I, P]
            L.orc_gamma_for_frame.restype = D
            L.orc_gamma_for_frame.argtypes = [I, I]
            L.orc_uncertainty_points.argtypes = [P, P, I, P, I, D, P, I]
            L.orc_dq_from_rt.argtypes = [D, D, D, P]
            L.orc_rt_from_dq.argtypes = [P, P, P, P]
            L.orc_apply_warp.argtypes = [D, P, D, D, P]
            L.orc_field.argtypes = [P, P, P, I, I, I, I, I, D, P, I]
            L.orc_field_points.argtypes = [P, P, P, I, P, I, D, P, I]
            L.orc_mstep.argtypes = [P, P, P, I, D, P, P, P, P]
            L.orc_residuals.argtypes = [P, P, P, P, I, D, P]
            L.orc_fit.argtypes = [P, P, I, I, I, ctypes.POINTER(_Params), P, P, P, P, P, P, P, P]
            L.orc_warp.argtypes = [P, I, I, I, I, P, I, I, I, I, P, I, I, I, I, I]
            L.orc_insert_reference.argtypes = [P, I, I, I, I, P, I, I, I, I, I]
            L.orc_max_threads.restype = I
            _lib = L
    return _lib


def _d(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def max_threads() -> int:
    return lib().orc_max_threads()


def alpha_for_frame(w: int, h: int) -> float:
    return lib().orc_alpha_for_frame(int(w), int(h))


def dq_from_rt(th: float, tx: float, ty: float) -> np.ndarray:
    q = np.zeros(4)
    lib().orc_dq_from_rt(float(th), float(tx), float(ty), _p(q))
    return q


def rt_from_dq(q) -> tuple[float, float, float]:
    q = _d(q, (4,))
    out = [ctypes.c_double() for _ in range(3)]
    lib().orc_rt_from_dq(_p(q), *[ctypes.cast(ctypes.pointer(o), ctypes.c_void_p) for o in out])
    return tuple(o.value for o in out)


def apply_warp(s: float, q, px: float, py: float) -> np.ndarray:
    q = _d(q, (4,))
    out = np.zeros(2)
    lib().orc_apply_warp(float(s), _p(q), float(px), float(py), _p(out))
    return out


def field(q8, c, src, grid, alpha: float, nthreads: int = 0) -> np.ndarray:
    """Dense field on grid=(x0, y0, w, h); returns [h, w, 2] float64."""
    q8, c, src = _d(q8), _d(c), _d(src)
    n = c.shape[0]
    x0, y0, gw, gh = (int(v) for v in grid)
    out = np.empty((gh, gw, 2))
    rc = lib().orc_field(_p(q8), _p(c), _p(src), n, x0, y0, gw, gh, float(alpha), _p(out),
                         nthreads or max_threads())
    assert rc == OK, rc
    return out


def field_points(q8, c, src, pts, alpha: float, nthreads: int = 0) -> np.ndarray:
    q8, c, src, pts = _d(q8), _d(c), _d(src), _d(pts)
    out = np.empty((pts.shape[0], 2))
    rc = lib().orc_field_points(_p(q8), _p(c), _p(src), c.shape[0], _p(pts), pts.shape[0],
                                float(alpha), _p(out), nthreads or max_threads())
    assert rc == OK, rc
    return out


def beta_for_frame(w: int, h: int) -> float:
    return lib().orc_beta_for_frame(int(w), int(h))


def uncertainty(c, src, grid, beta: float, nthreads: int = 0) -> np.ndarray:
    """Eq. 8 on grid=(x0, y0, w, h): [h, w] float64, +inf where there is no inlier."""
    c, src = _d(c), _d(src)
    x0, y0, gw, gh = (int(v) for v in grid)
    out = np.empty((gh, gw))
    rc = lib().orc_uncertainty(_p(c), _p(src), c.shape[0], x0, y0, gw, gh, float(beta), _p(out),
                               nthreads or max_threads())
    assert rc == OK, rc
    return out


def uncertainty_points(c, src, pts, beta: float, nthreads: int = 0) -> np.ndarray:
    c, src, pts = _d(c), _d(src), _d(pts)
    out = np.empty(pts.shape[0])
    rc = lib().orc_uncertainty_points(_p(c), _p(src), c.shape[0], _p(pts), pts.shape[0],
                                      float(beta), _p(out), nthreads or max_threads())
    assert rc == OK, rc
    return out


def gamma_for_frame(w: int, h: int) -> float:
    return lib().orc_gamma_for_frame(int(w), int(h))


def compose(w_old, dw) -> np.ndarray:
    """App. A: the warp row w_new with s_new q_new(x) = ds dq(s_old q_old(x))."""
    w_old, dw = _d(w_old, (8,)), _d(dw, (8,))
    out = np.empty(8)
    lib().orc_compose(_p(w_old), _p(dw), _p(out))
    return out


def node_track(x0, w_old, s2_old, q8, c, src, alpha: float, beta: float, nthreads: int = 0):
    """Eq. 5 + App. A + Eq. 9 for every node: (w_new [nn, 8], s2_new [nn])."""
    x0, w_old, s2_old = _d(x0), _d(w_old), _d(s2_old)
    q8, c, src = _d(q8), _d(c), _d(src)
    nn = s2_old.shape[0]
    w_new, s2_new = np.empty((nn, 8)), np.empty(nn)
    rc = lib().orc_node_track(_p(x0), _p(w_old), _p(s2_old), nn, _p(q8), _p(c), _p(src),
                              c.shape[0], float(alpha), float(beta), _p(w_new), _p(s2_new),
                              nthreads or max_threads())
    assert rc == OK, rc
    return w_new, s2_new


def node_merge(x0, w_track, s2_track, w_loop, s2_loop, w_key, gamma: float):
    """Eqs. 12-15 for every node: (w_out [nn, 8], s2_out [nn])."""
    x0, w_track, s2_track = _d(x0), _d(w_track), _d(s2_track)
    w_loop, s2_loop, w_key = _d(w_loop), _d(s2_loop), _d(w_key)
    nn = s2_track.shape[0]
    w_out, s2_out = np.empty((nn, 8)), np.empty(nn)
    rc = lib().orc_node_merge(_p(x0), _p(w_track), _p(s2_track), _p(w_loop), _p(s2_loop),
                              _p(w_key), nn, float(gamma), _p(w_out), _p(s2_out))
    assert rc == OK, rc
    return w_out, s2_out


def arap_smooth(x0, w_merge, s2, alpha: float, max_iters: int = 5):
    """Sec. III-D: ARAP-smoothed node warps [nn, 8] and the cost of every iteration run."""
    x0, w_merge, s2 = _d(x0), _d(w_merge), _d(s2)
    nn = s2.shape[0]
    w_out = np.empty((nn, 8))
    costs = np.full(max(1, max_iters), np.nan)
    rc = lib().orc_arap_smooth(_p(x0), _p(w_merge), _p(s2), nn, float(alpha), int(max_iters),
                               _p(w_out), _p(costs))
    assert rc == OK, rc
    return w_out, costs[:max_iters]


def arap_fit(x0, xt, alpha: float):
    """Sec. III-D, Eqs. 16-17 and ARAP1-3: every node's ARAP warp from the motion x0 -> xt."""
    x0, xt = _d(x0), _d(xt)
    nn = x0.shape[0]
    s, th, t, q8 = np.empty(nn), np.empty(nn), np.empty((nn, 2)), np.empty((nn, 8))
    rc = lib().orc_arap_fit(_p(x0), _p(xt), nn, float(alpha), _p(s), _p(th), _p(t), _p(q8))
    return dict(s=s, theta=th, t=t, q8=q8, status=rc)


def feature_uncertainty(src, dst, q8, c, alpha: float, beta: float, s2_prev) -> np.ndarray:
    """Eq. 10: the features' uncertainties after one EMDQ."""
    src, dst, q8, c, s2_prev = _d(src), _d(dst), _d(q8), _d(c), _d(s2_prev)
    out = np.empty(c.shape[0])
    rc = lib().orc_feature_uncertainty(_p(src), _p(dst), c.shape[0], _p(q8), _p(c), float(alpha),
                                       float(beta), _p(s2_prev), _p(out))
    assert rc == OK, rc
    return out


def node_init(x0, w, pts, alpha: float) -> np.ndarray:
    """Sec. III-E: warps [npts, 8] of new nodes at pts from the existing nodes (x0, w)."""
    x0, w, pts = _d(x0), _d(w), _d(pts)
    out = np.empty((pts.shape[0], 8))
    rc = lib().orc_node_init(_p(x0), _p(w), x0.shape[0], _p(pts), pts.shape[0], float(alpha), _p(out))
    assert rc == OK, rc
    return out


def hex_nodes(w: int, h: int, spacing: float) -> np.ndarray:
    """Sec. III-E's node set ("until all image areas are covered"), written as its definition:
    every point of the hexagonal lattice through the image centre ((w-1)/2, (h-1)/2) with the
    given spacing (rows spacing*sqrt(3)/2 apart, alternate rows shifted by spacing/2) that lies
    within the lattice's covering radius spacing/sqrt(3) of the frame [0, w-1] x [0, h-1], so
    every pixel has a node within that radius."""
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
    dy = spacing * np.sqrt(3.0) / 2.0
    m = spacing / np.sqrt(3.0)
    pts = []
    rmax = int(np.ceil(max(w, h) / dy)) + 2
    cmax = int(np.ceil(max(w, h) / spacing)) + 2
    for r in range(-rmax, rmax + 1):
        y = cy + r * dy
        off = 0.5 * spacing if r % 2 else 0.0
        for k in range(-cmax, cmax + 1):
            x = cx + off + k * spacing
            ex = max(0.0 - x, 0.0, x - (w - 1))
            ey = max(0.0 - y, 0.0, y - (h - 1))
            if ex * ex + ey * ey <= m * m:
                pts.append((x, y))
    return np.array(pts)


def node_restrict(x, s2, y, s2f, beta: float) -> np.ndarray:
    """Eq. 11: node uncertainties bounded by the features'."""
    x, s2, y, s2f = _d(x), _d(s2), _d(y), _d(s2f)
    out = np.empty(s2.shape[0])
    rc = lib().orc_node_restrict(_p(x), _p(s2), s2.shape[0], _p(y), _p(s2f), s2f.shape[0],
                                 float(beta), _p(out))
    assert rc == OK, rc
    return out


def keyframe_distances(xt, xk) -> np.ndarray:
    """Eq. 6: (1/N) sum_i |x_i,t - x_i,k| for every key frame k (xk: [nk, nn, 2])."""
    xt, xk = _d(xt), _d(xk)
    out = np.empty(xk.shape[0])
    rc = lib().orc_keyframe_distances(_p(xt), _p(xk), xt.shape[0], xk.shape[0], _p(out))
    assert rc == OK, rc
    return out


def mstep(src, dst, p, alpha: float):
    src, dst, p = _d(src), _d(dst), _d(p)
    n = p.shape[0]
    s, th, t, q8 = np.empty(n), np.empty(n), np.empty((n, 2)), np.empty((n, 8))
    rc = lib().orc_mstep(_p(src), _p(dst), _p(p), n, float(alpha), _p(s), _p(th), _p(t), _p(q8))
    return dict(s=s, theta=th, t=t, q8=q8, status=rc)


def residuals(src, dst, p, q8, alpha: float) -> np.ndarray:
    src, dst, p, q8 = _d(src), _d(dst), _d(p), _d(q8)
    e = np.empty(p.shape[0])
    rc = lib().orc_residuals(_p(src), _p(dst), _p(p), _p(q8), p.shape[0], float(alpha), _p(e))
    assert rc == OK, rc
    return e


def fit(src, dst, frame_w: int, frame_h: int, alpha: float = 0.0, max_iters: int = 20,
        tol_p: float = 1e-3, sigma2_floor: float = 0.25, p0=None) -> dict:
    src, dst = _d(src), _d(dst)
    n = src.shape[0]
    prm = _Params(float(alpha), int(max_iters), float(tol_p), float(sigma2_floor))
    q8, c, p = np.empty((n, 8)), np.empty(n), np.empty(n)
    trace = np.full(max(1, max_iters), np.nan)
    iters, s2, g = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    p0a = _d(p0) if p0 is not None else None
    rc = lib().orc_fit(_p(src), _p(dst), n, int(frame_w), int(frame_h), ctypes.byref(prm),
                       _p(p0a) if p0a is not None else None, _p(q8), _p(c), _p(p),
                       ctypes.cast(ctypes.byref(iters), ctypes.c_void_p),
                       ctypes.cast(ctypes.byref(s2), ctypes.c_void_p),
                       ctypes.cast(ctypes.byref(g), ctypes.c_void_p), _p(trace))
    return dict(q8=q8, c=c, p=p, iters=iters.value, sigma2=s2.value, gamma=g.value,
                dp_trace=trace[:iters.value].copy(), status=rc)


def _pitched(frame: np.ndarray):
    """(uint8 [fh, fw, ch] array, row pitch in bytes): a view whose rows are tight but lie
    further apart (a frame inside a wider buffer) keeps its pitch; anything else is copied."""
    frame = np.asarray(frame)
    if frame.ndim == 2:
        frame = frame[:, :, None]
    fh, fw, ch = frame.shape
    if (frame.dtype == np.uint8 and frame.strides[2] == 1 and frame.strides[1] == ch and
            frame.strides[0] >= fw * ch):
        return frame, frame.strides[0]
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    return frame, fw * ch


def warp(frame: np.ndarray, disp: np.ndarray, grid, canvas: np.ndarray, origin) -> int:
    """Blend one frame into canvas (uint8 [CH, CW, 4], modified in place)."""
    frame, pitch = _pitched(frame)
    fh, fw, ch = frame.shape
    disp = np.ascontiguousarray(disp, dtype=np.float32)
    assert canvas.dtype == np.uint8 and canvas.flags.c_contiguous and canvas.shape[2] == 4
    x0, y0, gw, gh = (int(v) for v in grid)
    return lib().orc_warp(_p(frame), fw, fh, ch, pitch, _p(disp), x0, y0, gw, gh,
                          _p(canvas), canvas.shape[1], canvas.shape[0], canvas.shape[1] * 4,
                          int(origin[0]), int(origin[1]))


def insert_reference(frame: np.ndarray, canvas: np.ndarray, origin) -> int:
    frame, pitch = _pitched(frame)
    fh, fw, ch = frame.shape
    return lib().orc_insert_reference(_p(frame), fw, fh, ch, pitch, _p(canvas),
                                      canvas.shape[1], canvas.shape[0], canvas.shape[1] * 4,
                                      int(origin[0]), int(origin[1]))
