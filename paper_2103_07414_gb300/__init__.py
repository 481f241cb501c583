"""GB300-native EMDQ dense deformation field and mosaic warp (arXiv 2103.07414).

A thin binding over the C ABI of ``libemdq.so`` (declared in ``include/emdq.h``): it
checks tensor devices, dtypes and layouts, allocates outputs and workspaces with torch,
and passes raw device pointers and the current CUDA stream.  Every step of the path runs
in the library's CUDA kernels; there is no CPU or PyTorch fallback -- if the library is
missing or a CUDA device is not available, these functions raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from ._build import LIB as _LIB_PATH, build  # noqa: F401

__all__ = ['emdq_fit', 'emdq_fit_batch', 'emdq_field', 'emdq_field_batch', 'field_batch_autotune',
           'field_batch_tile_rows', 'emdq_mosaic_batch', 'mosaic_batch_workspace_size', 'mosaic_warp',
           'mosaic_warp_batch', 'emdq_batch', 'emdq_mosaic_pairs', 'mosaic_pairs_workspace_size', 'emdq_mosaic', 'emdq_uncertainty', 'node_track', 'node_merge', 'node_restrict', 'feature_uncertainty',
           'keyframe_distances', 'hex_nodes', 'node_init', 'arap_smooth',
           'mosaic_insert_reference',
           'alpha_for_frame', 'fit_workspace_size', 'field_workspace_size', 'EmdqError',
           'FP32', 'BF16', 'STATUS', 'lib', 'build']

FP32, BF16 = 0, 1
STATUS = {0: 'OK', 1: 'EINVAL', 2: 'EDEGENERATE', 3: 'ENOCONV', 4: 'ETIMEOUT', 5: 'ECUDA',
          6: 'EWORKSPACE', 7: 'ENOTSUP', 8: 'ENONFINITE'}


class EmdqError(RuntimeError):
    def __init__(self, where: str, code: int):
        self.code = code
        super().__init__(f'{where}: {STATUS.get(code, code)} ({lib().emdq_status_string(code).decode()})')


class _Params(ctypes.Structure):
    _fields_ = [('alpha', ctypes.c_float), ('max_iters', ctypes.c_int),
                ('tol_p', ctypes.c_float), ('sigma2_floor', ctypes.c_float),
                ('reserved', ctypes.c_int * 4)]


class _MosaicFrame(ctypes.Structure):
    _fields_ = [('frame', ctypes.c_void_p), ('disp', ctypes.c_void_p), ('grid_x0', ctypes.c_int),
                ('grid_y0', ctypes.c_int), ('grid_w', ctypes.c_int), ('grid_h', ctypes.c_int)]


class _FieldProblem(ctypes.Structure):
    _fields_ = [('q', ctypes.c_void_p), ('c', ctypes.c_void_p), ('src', ctypes.c_void_p),
                ('n', ctypes.c_int), ('grid_x0', ctypes.c_int), ('grid_y0', ctypes.c_int),
                ('grid_w', ctypes.c_int), ('grid_h', ctypes.c_int), ('alpha', ctypes.c_float),
                ('disp_out', ctypes.c_void_p)]


class _MosaicPair(ctypes.Structure):
    _fields_ = [('q', ctypes.c_void_p), ('c', ctypes.c_void_p), ('src', ctypes.c_void_p),
                ('n', ctypes.c_int), ('grid_x0', ctypes.c_int), ('grid_y0', ctypes.c_int),
                ('grid_w', ctypes.c_int), ('grid_h', ctypes.c_int), ('alpha', ctypes.c_float),
                ('frame', ctypes.c_void_p), ('fw', ctypes.c_int), ('fh', ctypes.c_int),
                ('frame_pitch', ctypes.c_int), ('canvas', ctypes.c_void_p), ('canvas_w', ctypes.c_int),
                ('canvas_h', ctypes.c_int), ('canvas_pitch', ctypes.c_int), ('origin_x', ctypes.c_int),
                ('origin_y', ctypes.c_int)]


class _MosaicProblem(ctypes.Structure):
    _fields_ = [('q', ctypes.c_void_p), ('c', ctypes.c_void_p), ('src', ctypes.c_void_p),
                ('n', ctypes.c_int), ('grid_x0', ctypes.c_int), ('grid_y0', ctypes.c_int),
                ('grid_w', ctypes.c_int), ('grid_h', ctypes.c_int), ('alpha', ctypes.c_float),
                ('frame', ctypes.c_void_p)]


class _Pair(ctypes.Structure):
    _fields_ = [('src', ctypes.c_void_p), ('dst', ctypes.c_void_p), ('n', ctypes.c_int),
                ('frame_w', ctypes.c_int), ('frame_h', ctypes.c_int), ('frame', ctypes.c_void_p),
                ('channels', ctypes.c_int), ('frame_pitch', ctypes.c_int), ('grid_x0', ctypes.c_int),
                ('grid_y0', ctypes.c_int), ('grid_w', ctypes.c_int), ('grid_h', ctypes.c_int),
                ('canvas', ctypes.c_void_p), ('canvas_w', ctypes.c_int), ('canvas_h', ctypes.c_int),
                ('canvas_pitch', ctypes.c_int), ('origin_x', ctypes.c_int), ('origin_y', ctypes.c_int),
                ('q_out', ctypes.c_void_p), ('c_out', ctypes.c_void_p), ('p_out', ctypes.c_void_p),
                ('info', ctypes.c_void_p)]


class _Problem(ctypes.Structure):
    _fields_ = [('src', ctypes.c_void_p), ('dst', ctypes.c_void_p), ('n', ctypes.c_int),
                ('frame_w', ctypes.c_int), ('frame_h', ctypes.c_int), ('p0', ctypes.c_void_p),
                ('q_out', ctypes.c_void_p), ('c_out', ctypes.c_void_p), ('p_out', ctypes.c_void_p),
                ('info', ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load libemdq.so (built in-tree by ``build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f'libemdq.so not built ({_LIB_PATH}); run '
                                   'paper_2103_07414_gb300.build() first')
            L = ctypes.CDLL(_LIB_PATH)
            P, I, F, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
            L.emdq_default_params.argtypes = [ctypes.POINTER(_Params)]
            L.emdq_alpha_for_frame.restype = F
            L.emdq_alpha_for_frame.argtypes = [I, I]
            L.emdq_status_string.restype = ctypes.c_char_p
            L.emdq_status_string.argtypes = [I]
            L.emdq_abi_version.restype = I
            L.emdq_fit_max_n.restype = I
            L.emdq_fit_workspace_size.restype = Z
            L.emdq_fit_workspace_size.argtypes = [I]
            L.emdq_fit.restype = I
            L.emdq_fit.argtypes = [P, P, I, I, I, ctypes.POINTER(_Params), P, P, P, P, P, P, Z, P]
            L.emdq_fit_batch_workspace_size.restype = Z
            L.emdq_fit_batch_workspace_size.argtypes = [P, I]
            L.emdq_fit_batch.restype = I
            L.emdq_fit_batch.argtypes = [P, I, ctypes.POINTER(_Params), P, Z, P]
            L.emdq_fit_batch_ex.restype = I
            L.emdq_fit_batch_ex.argtypes = [P, I, ctypes.POINTER(_Params), P, P, Z, P]
            L.emdq_fit_batch_phases.restype = I
            L.emdq_fit_batch_phases.argtypes = [P, I, ctypes.POINTER(_Params), P, I, P, Z, P]
            L.emdq_fit_batch_capacity.restype = I
            L.emdq_fit_batch_capacity.argtypes = [P, I]
            L.emdq_fit_batch_autotune.restype = I
            L.emdq_fit_batch_autotune.argtypes = [P, I, ctypes.POINTER(_Params), P, Z, P, I, P,
                                                  ctypes.POINTER(ctypes.c_float)]
            L.emdq_field_workspace_size.restype = Z
            L.emdq_field_workspace_size.argtypes = [I, I, I, I]
            L.emdq_field_batch_workspace_size.restype = Z
            L.emdq_field_batch_workspace_size.argtypes = [P, I]
            L.emdq_field_batch.restype = I
            L.emdq_field_batch.argtypes = [P, I, P, Z, P]
            L.emdq_field_batch_ex.restype = I
            L.emdq_field_batch_ex.argtypes = [P, I, I, P, Z, P]
            L.emdq_field_batch_tile_rows.restype = I
            L.emdq_field_batch_tile_rows.argtypes = [P, I]
            L.emdq_field_batch_autotune.restype = I
            L.emdq_field_batch_autotune.argtypes = [P, I, P, Z, P, I, P, P]
            L.emdq_mosaic_batch_workspace_size.restype = Z
            L.emdq_mosaic_batch_workspace_size.argtypes = [P, I]
            L.emdq_mosaic_batch_ex.restype = I
            L.emdq_mosaic_batch_ex.argtypes = [P, I, I, I, I, I, P, I, I, I, I, I, I, P, Z, P]
            L.emdq_mosaic_batch.restype = I
            L.emdq_mosaic_pairs_workspace_size.restype = Z
            L.emdq_mosaic_pairs_workspace_size.argtypes = [P, I]
            L.emdq_mosaic_pairs.restype = I
            L.emdq_mosaic_pairs.argtypes = [P, I, I, P, Z, P]
            L.emdq_mosaic_batch.argtypes = [P, I, I, I, I, I, P, I, I, I, I, I, P, Z, P]
            L.emdq_field.restype = I
            L.emdq_field.argtypes = [P, P, P, I, I, I, I, I, F, I, P, P, Z, P]
            L.mosaic_warp_batch.restype = I
            L.emdq_beta_for_frame.restype = F
            L.emdq_beta_for_frame.argtypes = [I, I]
            L.emdq_uncertainty.argtypes = [P, P, I, I, I, I, I, F, P, P]
            L.emdq_gamma_for_frame.restype = F
            L.emdq_gamma_for_frame.argtypes = [I, I]
            L.emdq_node_track.argtypes = [P, P, P, I, P, P, P, I, F, F, P, P, P]
            L.emdq_node_merge.argtypes = [P, P, P, P, P, P, I, F, P, P, P]
            L.emdq_arap_workspace_size.argtypes = [I]
            L.emdq_arap_workspace_size.restype = Z
            L.emdq_arap_smooth.argtypes = [P, P, P, I, F, I, P, P, Z, P]
            L.emdq_node_restrict.argtypes = [P, P, I, P, P, I, F, P, P]
            L.emdq_hex_nodes.argtypes = [I, I, F, P, I]
            L.emdq_hex_nodes.restype = I
            L.emdq_node_init.argtypes = [P, P, I, P, I, F, P, P]
            L.emdq_feature_uncertainty.argtypes = [P, P, I, P, P, F, F, P, P, P]
            L.emdq_keyframe_distances.argtypes = [P, P, I, I, P, P]
            L.emdq_batch_workspace_size.argtypes = [P, I, I]
            L.emdq_batch_workspace_size.restype = Z
            L.emdq_batch.argtypes = [P, I, ctypes.POINTER(_Params), P, P, P, Z, P]
            L.emdq_batch_ex.restype = I
            L.emdq_batch_ex.argtypes = [P, I, ctypes.POINTER(_Params), P, P, P, I, P, Z, P]
            L.mosaic_warp_batch.argtypes = [P, I, I, I, I, I, P, I, I, I, I, I, P]
            L.mosaic_warp.restype = I
            L.mosaic_warp.argtypes = [P, I, I, I, I, P, I, I, I, I, P, I, I, I, I, I, P]
            L.emdq_mosaic.restype = I
            L.emdq_mosaic.argtypes = [P, P, P, I, I, I, I, I, F, P, I, I, I, I, P, I, I, I, I, I,
                                      P, Z, P]
            L.emdq_mlp_param_count.restype = I
            L.emdq_warm_features.restype = I
            L.emdq_warm_features.argtypes = [P, P, I, P, P]
            L.emdq_warm_infer.restype = I
            L.emdq_warm_infer.argtypes = [P, I, P, P, P]
            L.emdq_warm_start.restype = I
            L.emdq_warm_start.argtypes = [P, P, P, P, I, P, P]
            L.emdq_mlp_train_workspace_size.restype = Z
            L.emdq_mlp_train_workspace_size.argtypes = [I]
            L.emdq_mlp_train_step.restype = I
            L.emdq_mlp_train_step.argtypes = [P, P, I, P, P, P, I, F, P, P, P, Z, P]
            L.mosaic_insert_reference.restype = I
            L.mosaic_insert_reference.argtypes = [P, I, I, I, I, P, I, I, I, I, I, P]
            _lib = L
    return _lib


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(t: torch.Tensor, name: str, dtype: torch.dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f'{name} must be a CUDA tensor')
    if t.dtype != dtype:
        raise ValueError(f'{name} must be {dtype}, got {t.dtype}')
    if not t.is_contiguous():
        raise ValueError(f'{name} must be contiguous')
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f'{name} must have shape {tuple(shape)}, got {tuple(t.shape)}')


def alpha_for_frame(w: int, h: int) -> float:
    return lib().emdq_alpha_for_frame(int(w), int(h))


def beta_for_frame(w: int, h: int) -> float:
    return lib().emdq_beta_for_frame(int(w), int(h))


def fit_workspace_size(n: int) -> int:
    return lib().emdq_fit_workspace_size(int(n))


def field_workspace_size(n: int, grid_w: int, grid_h: int, precision: int) -> int:
    return lib().emdq_field_workspace_size(int(n), int(grid_w), int(grid_h), int(precision))


def _workspace(nbytes: int, device, given: torch.Tensor | None) -> torch.Tensor:
    if given is not None:
        _check(given, 'workspace', torch.uint8)
        return given
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def emdq_fit(src: torch.Tensor, dst: torch.Tensor, frame_w: int, frame_h: int, *,
             alpha: float = 0.0, max_iters: int = 20, tol_p: float = 1e-3,
             sigma2_floor: float = 0.25, p0: torch.Tensor | None = None,
             out: dict | None = None, workspace: torch.Tensor | None = None, stream=None,
             reserved=(0, 0, 0, 0)) -> dict:
    """EMDQ fit of n matches (src, dst: [n, 2] float32 CUDA).  Returns dict with q [n, 8],
    c [n], p [n] and info [4] (int32 view: status, iters; float view: sigma2, gamma).
    reserved: emdq_params.reserved (the bounded waits' settings)."""
    n = src.shape[0]
    _check(src, 'src', torch.float32, (n, 2))
    _check(dst, 'dst', torch.float32, (n, 2))
    if p0 is not None:
        _check(p0, 'p0', torch.float32, (n,))
    dev = src.device
    o = out if out is not None else {}
    q = o.get('q') if o.get('q') is not None else torch.empty((n, 8), dtype=torch.float32, device=dev)
    c = o.get('c') if o.get('c') is not None else torch.empty(n, dtype=torch.float32, device=dev)
    p = o.get('p') if o.get('p') is not None else torch.empty(n, dtype=torch.float32, device=dev)
    info = o.get('info') if o.get('info') is not None else torch.zeros(4, dtype=torch.int32, device=dev)
    ws = _workspace(fit_workspace_size(n), dev, workspace)
    prm = _Params(float(alpha), int(max_iters), float(tol_p), float(sigma2_floor),
                  (ctypes.c_int * 4)(*reserved))
    rc = lib().emdq_fit(_ptr(src), _ptr(dst), n, int(frame_w), int(frame_h), ctypes.byref(prm),
                        _ptr(p0), _ptr(q), _ptr(c), _ptr(p), _ptr(info), _ptr(ws), ws.numel(),
                        _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_fit', rc)
    return dict(q=q, c=c, p=p, info=info, workspace=ws)


def _batch_args(problems, outs):
    count = len(problems)
    arr = (_Problem * max(1, count))()
    results = []
    for b, pr in enumerate(problems):
        src, dst, fw, fh = pr[:4]
        p0 = pr[4] if len(pr) > 4 else None
        n = src.shape[0]
        _check(src, 'src', torch.float32, (n, 2))
        _check(dst, 'dst', torch.float32, (n, 2))
        if p0 is not None:
            _check(p0, 'p0', torch.float32, (n,))
        o = outs[b] if outs is not None else {}
        dev = src.device
        r = dict(q=o.get('q') if o.get('q') is not None else torch.empty((n, 8), device=dev),
                 c=o.get('c') if o.get('c') is not None else torch.empty(n, device=dev),
                 p=o.get('p') if o.get('p') is not None else torch.empty(n, device=dev),
                 info=o.get('info') if o.get('info') is not None else
                 torch.zeros(4, dtype=torch.int32, device=dev))
        arr[b] = _Problem(src.data_ptr(), dst.data_ptr(), n, int(fw), int(fh),
                          p0.data_ptr() if p0 is not None else None, r['q'].data_ptr(),
                          r['c'].data_ptr(), r['p'].data_ptr(), r['info'].data_ptr())
        results.append(r)
    return arr, results


def emdq_fit_batch(problems, *, alpha: float = 0.0, max_iters: int = 20, tol_p: float = 1e-3,
                   sigma2_floor: float = 0.25, outs: list | None = None,
                   workspace: torch.Tensor | None = None, ctas=None, stream=None,
                   reserved=(0, 0, 0, 0), phases=None) -> list:
    """Fit several independent problems in one launch.  problems: list of
    (src, dst, frame_w, frame_h) or (src, dst, frame_w, frame_h, p0).  ctas: optional CTAs per
    problem (default: in proportion to n^2).  phases: increasing EM round counts for
    emdq_fit_batch_phases (the last one replaces max_iters; not with ctas).  Returns one dict
    per problem as emdq_fit does."""
    count = len(problems)
    arr, results = _batch_args(problems, outs)
    need = lib().emdq_fit_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), count)
    dev = problems[0][0].device
    ws = _workspace(need, dev, workspace)
    prm = _Params(float(alpha), int(max_iters), float(tol_p), float(sigma2_floor),
                  (ctypes.c_int * 4)(*reserved))
    if phases is not None:
        if ctas is not None:
            raise ValueError('phases and ctas: one or the other')
        ph = (ctypes.c_int * max(1, len(phases)))(*[int(v) for v in phases])
        rc = lib().emdq_fit_batch_phases(ctypes.cast(arr, ctypes.c_void_p), count, ctypes.byref(prm),
                                         ctypes.cast(ph, ctypes.c_void_p), len(phases), _ptr(ws),
                                         ws.numel(), _stream(stream))
        if rc != 0:
            raise EmdqError('emdq_fit_batch_phases', rc)
        return results
    split = None
    if ctas is not None:
        if len(ctas) != count:
            raise ValueError('ctas: one entry per problem')
        split = (ctypes.c_int * count)(*[int(v) for v in ctas])
    rc = lib().emdq_fit_batch_ex(ctypes.cast(arr, ctypes.c_void_p), count, ctypes.byref(prm),
                                 ctypes.cast(split, ctypes.c_void_p) if split is not None else None,
                                 _ptr(ws), ws.numel(), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_fit_batch', rc)
    return results


def fit_batch_capacity(problems) -> int:
    """Co-resident CTAs of the batch kernel for these problems."""
    count = len(problems)
    arr = (_Problem * max(1, count))()
    for b, pr in enumerate(problems):
        arr[b].n = int(pr[0].shape[0])
    return lib().emdq_fit_batch_capacity(ctypes.cast(arr, ctypes.c_void_p), count)


def fit_batch_autotune(problems, *, reps: int = 3, alpha: float = 0.0, max_iters: int = 20,
                       tol_p: float = 1e-3, sigma2_floor: float = 0.25, outs: list | None = None,
                       workspace: torch.Tensor | None = None, stream=None):
    """Time the candidate CTA splits of the library's autotuner on these problems; returns
    (ctas per problem, best ms).  Synchronises; not inside a stream capture."""
    count = len(problems)
    arr, _ = _batch_args(problems, outs)
    need = lib().emdq_fit_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), count)
    ws = _workspace(need, problems[0][0].device, workspace)
    prm = _Params(float(alpha), int(max_iters), float(tol_p), float(sigma2_floor), (ctypes.c_int * 4)())
    out = (ctypes.c_int * count)()
    ms = ctypes.c_float(0.0)
    rc = lib().emdq_fit_batch_autotune(ctypes.cast(arr, ctypes.c_void_p), count, ctypes.byref(prm),
                                       _ptr(ws), ws.numel(), _stream(stream), int(reps),
                                       ctypes.cast(out, ctypes.c_void_p), ctypes.byref(ms))
    if rc != 0:
        raise EmdqError('emdq_fit_batch_autotune', rc)
    return [int(v) for v in out], float(ms.value)


def fit_batch_workspace_size(problems) -> int:
    count = len(problems)
    arr = (_Problem * max(1, count))()
    for b, pr in enumerate(problems):
        arr[b].n = int(pr[0].shape[0])
    return lib().emdq_fit_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), count)


def read_fit_info(info: torch.Tensor) -> dict:
    """Decode the 16-byte device record (synchronises with its stream)."""
    h = info.cpu()
    iv = h.view(torch.int32)
    fv = h.view(torch.float32)
    return dict(status=int(iv[0]), status_name=STATUS.get(int(iv[0]), '?'), iters=int(iv[1]),
                sigma2=float(fv[2]), gamma=float(fv[3]))


def emdq_field(q: torch.Tensor, c: torch.Tensor, src: torch.Tensor, grid, alpha: float, *,
               precision: int = BF16, out: torch.Tensor | None = None,
               workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Dense displacement on grid=(x0, y0, w, h): returns [h, w, 2] float32 CUDA."""
    n = c.shape[0]
    _check(q, 'q', torch.float32, (n, 8))
    _check(c, 'c', torch.float32, (n,))
    _check(src, 'src', torch.float32, (n, 2))
    x0, y0, gw, gh = (int(v) for v in grid)
    if out is None:
        out = torch.empty((gh, gw, 2), dtype=torch.float32, device=q.device)
    _check(out, 'out', torch.float32, (gh, gw, 2))
    ws = _workspace(field_workspace_size(n, gw, gh, precision), q.device, workspace)
    rc = lib().emdq_field(_ptr(q), _ptr(c), _ptr(src), n, x0, y0, gw, gh, float(alpha),
                          int(precision), _ptr(out), _ptr(ws), ws.numel(), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_field', rc)
    return out


def _field_problems(problems, outs):
    count = len(problems)
    arr = (_FieldProblem * max(1, count))()
    res = []
    for b, (q, c, src, grid, alpha) in enumerate(problems):
        n = c.shape[0]
        _check(q, 'q', torch.float32, (n, 8))
        _check(c, 'c', torch.float32, (n,))
        _check(src, 'src', torch.float32, (n, 2))
        x0, y0, gw, gh = (int(v) for v in grid)
        out = outs[b] if outs is not None else torch.empty((gh, gw, 2), dtype=torch.float32,
                                                           device=q.device)
        _check(out, 'out', torch.float32, (gh, gw, 2))
        arr[b] = _FieldProblem(_ptr(q), _ptr(c), _ptr(src), n, x0, y0, gw, gh, float(alpha), _ptr(out))
        res.append(out)
    return arr, res


def field_batch_workspace_size(problems) -> int:
    """Bytes of workspace for emdq_field_batch on (q, c, src, grid, alpha) problems."""
    arr = (_FieldProblem * max(1, len(problems)))()
    for b, (q, c, src, grid, alpha) in enumerate(problems):
        arr[b].n = int(c.shape[0])
        arr[b].grid_w, arr[b].grid_h = int(grid[2]), int(grid[3])
    return lib().emdq_field_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), len(problems))


def emdq_field_batch(problems, *, outs: list | None = None, workspace: torch.Tensor | None = None,
                     stream=None, tile_rows: int | None = None) -> list:
    """BF16 fields of several (q, c, src, grid, alpha) problems in one operand launch and one
    persistent tensor-core launch; returns the [h, w, 2] fields (or fills outs).  tile_rows:
    the GEMM's tile height (16, 24, 32 or 40); default: the autotuned or built-in choice."""
    count = len(problems)
    arr, res = _field_problems(problems, outs)
    need = lib().emdq_field_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), count)
    ws = _workspace(need, problems[0][0].device, workspace)
    if tile_rows is None:
        rc = lib().emdq_field_batch(ctypes.cast(arr, ctypes.c_void_p), count, _ptr(ws), ws.numel(),
                                    _stream(stream))
    else:
        rc = lib().emdq_field_batch_ex(ctypes.cast(arr, ctypes.c_void_p), count, int(tile_rows),
                                       _ptr(ws), ws.numel(), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_field_batch', rc)
    return res


def _mosaic_problems(problems):
    arr = (_MosaicProblem * max(1, len(problems)))()
    fargs = None
    for b, (q, c, src, grid, alpha, frame) in enumerate(problems):
        n = c.shape[0]
        _check(q, 'q', torch.float32, (n, 8))
        _check(c, 'c', torch.float32, (n,))
        _check(src, 'src', torch.float32, (n, 2))
        fa = _frame_args(frame)
        if fargs is not None and fa != fargs:
            raise ValueError('frames of one sequence: the same size, channels and pitch')
        fargs = fa
        x0, y0, gw, gh = (int(v) for v in grid)
        arr[b] = _MosaicProblem(_ptr(q), _ptr(c), _ptr(src), n, x0, y0, gw, gh, float(alpha), _ptr(frame))
    return arr, fargs


def mosaic_batch_workspace_size(problems) -> int:
    arr, _ = _mosaic_problems(problems)
    return lib().emdq_mosaic_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), len(problems))


def emdq_mosaic_batch(problems, canvas: torch.Tensor, origin, *, tile_rows: int | None = None,
                      workspace: torch.Tensor | None = None, stream=None) -> None:
    """BF16 field and mosaic update of a group of frames of one sequence in one pass:
    problems = [(q, c, src, grid, alpha, frame), ...] in frame order; the canvas ends bit for bit
    as after emdq_field_batch then mosaic_warp_batch."""
    count = len(problems)
    if count < 1:
        raise ValueError('at least one frame')
    arr, (fw, fh, ch, pitch) = _mosaic_problems(problems)
    _check(canvas, 'canvas', torch.uint8)
    if canvas.dim() != 3 or canvas.shape[2] != 4:
        raise ValueError('canvas must be [h, w, 4] uint8')
    need = lib().emdq_mosaic_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), count)
    if need == 0:
        raise EmdqError('emdq_mosaic_batch_workspace_size', 1)
    ws = _workspace(need, canvas.device, workspace)
    ox, oy = (int(v) for v in origin)
    args = [ctypes.cast(arr, ctypes.c_void_p), count, fw, fh, ch, pitch, _ptr(canvas), canvas.shape[1],
            canvas.shape[0], canvas.shape[1] * 4, ox, oy]
    if tile_rows is None:
        rc = lib().emdq_mosaic_batch(*args, _ptr(ws), ws.numel(), _stream(stream))
    else:
        rc = lib().emdq_mosaic_batch_ex(*args, int(tile_rows), _ptr(ws), ws.numel(), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_mosaic_batch', rc)


def _mosaic_pairs(pairs):
    arr = (_MosaicPair * max(1, len(pairs)))()
    chs = set()
    for b, (q, c, src, grid, alpha, frame, canvas, origin) in enumerate(pairs):
        n = c.shape[0]
        _check(q, 'q', torch.float32, (n, 8))
        _check(c, 'c', torch.float32, (n,))
        _check(src, 'src', torch.float32, (n, 2))
        fw, fh, ch, pitch = _frame_args(frame)
        chs.add(ch)
        _check(canvas, 'canvas', torch.uint8)
        if canvas.dim() != 3 or canvas.shape[2] != 4:
            raise ValueError('canvas must be [h, w, 4] uint8')
        x0, y0, gw, gh = (int(v) for v in grid)
        ox, oy = (int(v) for v in origin)
        arr[b] = _MosaicPair(_ptr(q), _ptr(c), _ptr(src), n, x0, y0, gw, gh, float(alpha), _ptr(frame),
                             fw, fh, pitch, _ptr(canvas), canvas.shape[1], canvas.shape[0],
                             canvas.shape[1] * 4, ox, oy)
    if len(chs) > 1:
        raise ValueError('every pair of one call needs the same channel count')
    return arr, (chs.pop() if chs else 1)


def mosaic_pairs_workspace_size(pairs) -> int:
    arr, _ = _mosaic_pairs(pairs)
    return lib().emdq_mosaic_pairs_workspace_size(ctypes.cast(arr, ctypes.c_void_p), len(pairs))


def emdq_mosaic_pairs(pairs, *, workspace: torch.Tensor | None = None, stream=None) -> None:
    """BF16 field and mosaic update of up to 16 independent pairs in one pass:
    pairs = [(q, c, src, grid, alpha, frame, canvas, origin), ...], each with its own frame and
    canvas; every canvas ends bit for bit as after emdq_field (BF16) then mosaic_warp."""
    count = len(pairs)
    if count < 1:
        raise ValueError('at least one pair')
    arr, ch = _mosaic_pairs(pairs)
    need = lib().emdq_mosaic_pairs_workspace_size(ctypes.cast(arr, ctypes.c_void_p), count)
    if need == 0:
        raise EmdqError('emdq_mosaic_pairs_workspace_size', 1)
    ws = _workspace(need, pairs[0][0].device, workspace)
    rc = lib().emdq_mosaic_pairs(ctypes.cast(arr, ctypes.c_void_p), count, ch, _ptr(ws), ws.numel(),
                                 _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_mosaic_pairs', rc)


def field_batch_tile_rows(problems) -> int:
    """The tile height emdq_field_batch uses for a batch like this one."""
    arr = (_FieldProblem * max(1, len(problems)))()
    for b, (q, c, src, grid, alpha) in enumerate(problems):
        arr[b].n = int(c.shape[0])
        arr[b].grid_w, arr[b].grid_h = int(grid[2]), int(grid[3])
    return lib().emdq_field_batch_tile_rows(ctypes.cast(arr, ctypes.c_void_p), len(problems))


def field_batch_autotune(problems, *, reps: int = 5, outs: list | None = None,
                         workspace: torch.Tensor | None = None, stream=None) -> tuple:
    """Time every tile height on this batch and record the fastest for its size class:
    returns (tile_rows, ms per call).  Synchronises the stream."""
    count = len(problems)
    arr, res = _field_problems(problems, outs)
    need = lib().emdq_field_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), count)
    ws = _workspace(need, problems[0][0].device, workspace)
    py, ms = ctypes.c_int(0), ctypes.c_float(0.0)
    rc = lib().emdq_field_batch_autotune(ctypes.cast(arr, ctypes.c_void_p), count, _ptr(ws), ws.numel(),
                                         _stream(stream), int(reps), ctypes.byref(py), ctypes.byref(ms))
    if rc != 0:
        raise EmdqError('emdq_field_batch_autotune', rc)
    return py.value, ms.value


def emdq_uncertainty(c: torch.Tensor, src: torch.Tensor, grid, beta: float, *,
                     out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Eq. 8 on grid=(x0, y0, w, h): min over the inliers (c > 0) of exp(beta d^2), [h, w]
    float32 CUDA (+inf without inliers or beyond the FP32 range)."""
    n = c.shape[0]
    _check(c, 'c', torch.float32, (n,))
    _check(src, 'src', torch.float32, (n, 2))
    x0, y0, gw, gh = (int(v) for v in grid)
    if out is None:
        out = torch.empty((gh, gw), dtype=torch.float32, device=c.device)
    _check(out, 'out', torch.float32, (gh, gw))
    rc = lib().emdq_uncertainty(_ptr(c), _ptr(src), n, x0, y0, gw, gh, float(beta), _ptr(out),
                                _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_uncertainty', rc)
    return out


def gamma_for_frame(w: int, h: int) -> float:
    return lib().emdq_gamma_for_frame(int(w), int(h))


def node_track(x0: torch.Tensor, w_old: torch.Tensor, s2_old: torch.Tensor, q: torch.Tensor,
               c: torch.Tensor, src: torch.Tensor, alpha: float, beta: float, stream=None):
    """Eq. 5 + App. A + Eq. 9 for nn nodes: returns (w_new [nn, 8], s2_new [nn])."""
    nn, n = x0.shape[0], c.shape[0]
    _check(x0, 'x0', torch.float32, (nn, 2))
    _check(w_old, 'w_old', torch.float32, (nn, 8))
    _check(s2_old, 's2_old', torch.float32, (nn,))
    _check(q, 'q', torch.float32, (n, 8))
    _check(c, 'c', torch.float32, (n,))
    _check(src, 'src', torch.float32, (n, 2))
    w_new = torch.empty_like(w_old)
    s2_new = torch.empty_like(s2_old)
    rc = lib().emdq_node_track(_ptr(x0), _ptr(w_old), _ptr(s2_old), nn, _ptr(q), _ptr(c), _ptr(src),
                               n, float(alpha), float(beta), _ptr(w_new), _ptr(s2_new), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_node_track', rc)
    return w_new, s2_new


def node_merge(x0: torch.Tensor, w_track: torch.Tensor, s2_track: torch.Tensor, w_loop: torch.Tensor,
               s2_loop: torch.Tensor, w_key: torch.Tensor, gamma: float, stream=None):
    """Eqs. 12-15 for nn nodes: returns (w_out [nn, 8], s2_out [nn])."""
    nn = x0.shape[0]
    _check(x0, 'x0', torch.float32, (nn, 2))
    for name, t, shape in (('w_track', w_track, (nn, 8)), ('w_loop', w_loop, (nn, 8)),
                           ('w_key', w_key, (nn, 8)), ('s2_track', s2_track, (nn,)),
                           ('s2_loop', s2_loop, (nn,))):
        _check(t, name, torch.float32, shape)
    w_out = torch.empty_like(w_track)
    s2_out = torch.empty_like(s2_track)
    rc = lib().emdq_node_merge(_ptr(x0), _ptr(w_track), _ptr(s2_track), _ptr(w_loop), _ptr(s2_loop),
                               _ptr(w_key), nn, float(gamma), _ptr(w_out), _ptr(s2_out), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_node_merge', rc)
    return w_out, s2_out


def node_restrict(x: torch.Tensor, s2: torch.Tensor, y: torch.Tensor, s2f: torch.Tensor,
                  beta: float, stream=None) -> torch.Tensor:
    """Eq. 11: node uncertainties bounded by the features' (positions at the same time)."""
    nn, m = x.shape[0], y.shape[0]
    _check(x, 'x', torch.float32, (nn, 2))
    _check(s2, 's2', torch.float32, (nn,))
    _check(y, 'y', torch.float32, (m, 2))
    _check(s2f, 's2f', torch.float32, (m,))
    out = torch.empty_like(s2)
    rc = lib().emdq_node_restrict(_ptr(x), _ptr(s2), nn, _ptr(y), _ptr(s2f), m, float(beta), _ptr(out),
                                  _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_node_restrict', rc)
    return out


def feature_uncertainty(src: torch.Tensor, dst: torch.Tensor, q: torch.Tensor, c: torch.Tensor,
                        alpha: float, beta: float, s2_prev: torch.Tensor, stream=None) -> torch.Tensor:
    """Eq. 10: the features' uncertainties [n] after the EMDQ of (src -> dst)."""
    n = c.shape[0]
    _check(src, 'src', torch.float32, (n, 2))
    _check(dst, 'dst', torch.float32, (n, 2))
    _check(q, 'q', torch.float32, (n, 8))
    _check(c, 'c', torch.float32, (n,))
    _check(s2_prev, 's2_prev', torch.float32, (n,))
    out = torch.empty_like(s2_prev)
    rc = lib().emdq_feature_uncertainty(_ptr(src), _ptr(dst), n, _ptr(q), _ptr(c), float(alpha),
                                        float(beta), _ptr(s2_prev), _ptr(out), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_feature_uncertainty', rc)
    return out


def keyframe_distances(xt: torch.Tensor, xk: torch.Tensor, stream=None) -> torch.Tensor:
    """Eq. 6: mean node distance [nk] to every key frame (xk: [nk, nn, 2])."""
    nn = xt.shape[0]
    _check(xt, 'xt', torch.float32, (nn, 2))
    nk = xk.shape[0]
    _check(xk, 'xk', torch.float32, (nk, nn, 2))
    out = torch.empty(nk, dtype=torch.float32, device=xt.device)
    rc = lib().emdq_keyframe_distances(_ptr(xt), _ptr(xk), nn, nk, _ptr(out), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_keyframe_distances', rc)
    return out


def hex_nodes(w: int, h: int, spacing: float) -> torch.Tensor:
    """Sec. III-E: the node lattice of a w x h frame ([nn, 2] float32, CPU, breadth-first from
    the centre)."""
    n = lib().emdq_hex_nodes(int(w), int(h), float(spacing), None, 0)
    if n < 0:
        raise ValueError('hex_nodes: bad arguments')
    out = torch.empty((n, 2), dtype=torch.float32)
    lib().emdq_hex_nodes(int(w), int(h), float(spacing), ctypes.c_void_p(out.data_ptr()), n)
    return out


def node_init(x0: torch.Tensor, w: torch.Tensor, pts: torch.Tensor, alpha: float,
              stream=None) -> torch.Tensor:
    """Sec. III-E: warps [npts, 8] of new nodes at pts from the existing nodes (x0, w)."""
    nn, npts = x0.shape[0], pts.shape[0]
    _check(x0, 'x0', torch.float32, (nn, 2))
    _check(w, 'w', torch.float32, (nn, 8))
    _check(pts, 'pts', torch.float32, (npts, 2))
    out = torch.empty((npts, 8), dtype=torch.float32, device=x0.device)
    rc = lib().emdq_node_init(_ptr(x0), _ptr(w), nn, _ptr(pts), npts, float(alpha), _ptr(out),
                              _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_node_init', rc)
    return out


def arap_smooth(x0: torch.Tensor, w_merge: torch.Tensor, s2: torch.Tensor, alpha: float,
                max_iters: int = 5, workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Sec. III-D: ARAP-smoothed node warps [nn, 8] (at most max_iters iterations)."""
    nn = x0.shape[0]
    _check(x0, 'x0', torch.float32, (nn, 2))
    _check(w_merge, 'w_merge', torch.float32, (nn, 8))
    _check(s2, 's2', torch.float32, (nn,))
    w_out = torch.empty_like(w_merge)
    need = lib().emdq_arap_workspace_size(nn)
    if need == 0:
        raise EmdqError('emdq_arap_workspace_size', 7)
    ws = _workspace(need, x0.device, workspace)
    rc = lib().emdq_arap_smooth(_ptr(x0), _ptr(w_merge), _ptr(s2), nn, float(alpha), int(max_iters),
                                _ptr(w_out), _ptr(ws), ws.numel(), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_arap_smooth', rc)
    return w_out


def _frame_args(frame: torch.Tensor):
    _check(frame, 'frame', torch.uint8)
    if frame.dim() == 2:
        fh, fw = frame.shape
        ch = 1
    elif frame.dim() == 3 and frame.shape[2] in (1, 3):
        fh, fw, ch = frame.shape
    else:
        raise ValueError('frame must be [h, w] or [h, w, 1|3] uint8')
    return fw, fh, ch, fw * ch


def mosaic_warp(frame: torch.Tensor, disp: torch.Tensor, grid, canvas: torch.Tensor, origin,
                stream=None) -> None:
    """Blend frame into canvas ([CH, CW, 4] uint8 CUDA) through the field disp."""
    fw, fh, ch, pitch = _frame_args(frame)
    x0, y0, gw, gh = (int(v) for v in grid)
    _check(disp, 'disp', torch.float32, (gh, gw, 2))
    _check(canvas, 'canvas', torch.uint8)
    if canvas.dim() != 3 or canvas.shape[2] != 4:
        raise ValueError('canvas must be [h, w, 4] uint8')
    chh, cw = canvas.shape[:2]
    rc = lib().mosaic_warp(_ptr(frame), fw, fh, ch, pitch, _ptr(disp), x0, y0, gw, gh,
                           _ptr(canvas), cw, chh, cw * 4, int(origin[0]), int(origin[1]),
                           _stream(stream))
    if rc != 0:
        raise EmdqError('mosaic_warp', rc)


def mosaic_warp_batch(frames, disps, grids, canvas: torch.Tensor, origin, stream=None) -> None:
    """Blend up to 8 frames (same size and channels) into canvas in one launch, each through
    its own field and window; the canvas ends as after mosaic_warp on each in order."""
    count = len(frames)
    if not (len(disps) == len(grids) == count) or count < 1:
        raise ValueError('one field and one window per frame')
    fw, fh, ch, pitch = _frame_args(frames[0])
    arr = (_MosaicFrame * count)()
    for k, (fr, d, g) in enumerate(zip(frames, disps, grids)):
        if _frame_args(fr) != (fw, fh, ch, pitch):
            raise ValueError('frames of one sequence: the same size and channels')
        x0, y0, gw, gh = (int(v) for v in g)
        _check(d, 'disp', torch.float32, (gh, gw, 2))
        arr[k] = _MosaicFrame(_ptr(fr), _ptr(d), x0, y0, gw, gh)
    _check(canvas, 'canvas', torch.uint8)
    if canvas.dim() != 3 or canvas.shape[2] != 4:
        raise ValueError('canvas must be [h, w, 4] uint8')
    chh, cw = canvas.shape[:2]
    rc = lib().mosaic_warp_batch(ctypes.cast(arr, ctypes.c_void_p), count, fw, fh, ch, pitch,
                                 _ptr(canvas), cw, chh, cw * 4, int(origin[0]), int(origin[1]),
                                 _stream(stream))
    if rc != 0:
        raise EmdqError('mosaic_warp_batch', rc)


def _pair_args(pairs, outs):
    count = len(pairs)
    arr = (_Pair * max(1, count))()
    results = []
    for b, pr in enumerate(pairs):
        src, dst, frame, canvas = pr['src'], pr['dst'], pr['frame'], pr['canvas']
        n = src.shape[0]
        _check(src, 'src', torch.float32, (n, 2))
        _check(dst, 'dst', torch.float32, (n, 2))
        fw, fh, ch, pitch = _frame_args(frame)
        _check(canvas, 'canvas', torch.uint8)
        if canvas.dim() != 3 or canvas.shape[2] != 4:
            raise ValueError('canvas must be [h, w, 4] uint8')
        chh, cw = canvas.shape[:2]
        x0, y0, gw, gh = (int(v) for v in pr['grid'])
        ox, oy = (int(v) for v in pr['origin'])
        o = outs[b] if outs is not None else {}
        dev = src.device
        r = dict(q=o.get('q') if o.get('q') is not None else torch.empty((n, 8), device=dev),
                 c=o.get('c') if o.get('c') is not None else torch.empty(n, device=dev),
                 p=o.get('p') if o.get('p') is not None else torch.empty(n, device=dev),
                 info=o.get('info') if o.get('info') is not None else
                 torch.zeros(4, dtype=torch.int32, device=dev))
        arr[b] = _Pair(src.data_ptr(), dst.data_ptr(), n, fw, fh, frame.data_ptr(), ch, pitch,
                       x0, y0, gw, gh, canvas.data_ptr(), cw, chh, cw * 4, ox, oy,
                       r['q'].data_ptr(), r['c'].data_ptr(), r['p'].data_ptr(), r['info'].data_ptr())
        results.append(r)
    return arr, results


def batch_workspace_size(pairs, warm: bool = False) -> int:
    """Bytes of workspace for emdq_batch on these pairs (with or without the warm start)."""
    arr, _ = _pair_args(pairs, None)
    return lib().emdq_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), len(pairs), int(warm))


def emdq_batch(pairs, *, warm_params: torch.Tensor | None = None, fit_ctas=None,
               alpha: float = 0.0, max_iters: int = 20, tol_p: float = 1e-3,
               sigma2_floor: float = 0.25, outs: list | None = None,
               workspace: torch.Tensor | None = None, stream=None, fit_phases=None) -> list:
    """The whole path for up to 64 independent pairs in one call: warm start (if
    warm_params), all fits in one launch, BF16 fields 16 pairs per launch pair, and each
    pair's warp into its canvas in list order.  pairs: dicts with src, dst ([n, 2] float32),
    frame ([h, w] or [h, w, 1|3] uint8), grid (x0, y0, w, h), canvas ([H, W, 4] uint8) and
    origin (x, y).  fit_phases: the fits in phases (emdq_batch_ex; not with fit_ctas).  Returns
    one dict per pair (q, c, p, info) as emdq_fit does."""
    count = len(pairs)
    arr, results = _pair_args(pairs, outs)
    if warm_params is not None:
        _check(warm_params, 'warm_params', torch.float32, (lib().emdq_mlp_param_count(),))
    need = lib().emdq_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), count,
                                           int(warm_params is not None))
    if need == 0:
        raise EmdqError('emdq_batch_workspace_size', 1)
    ws = _workspace(need, pairs[0]['src'].device, workspace)
    prm = _Params(float(alpha), int(max_iters), float(tol_p), float(sigma2_floor), (ctypes.c_int * 4)())
    split = None
    if fit_ctas is not None:
        if len(fit_ctas) != count:
            raise ValueError('fit_ctas: one entry per pair')
        split = (ctypes.c_int * count)(*[int(v) for v in fit_ctas])
    if fit_phases is not None:
        ph = (ctypes.c_int * max(1, len(fit_phases)))(*[int(v) for v in fit_phases])
        rc = lib().emdq_batch_ex(ctypes.cast(arr, ctypes.c_void_p), count, ctypes.byref(prm),
                                 _ptr(warm_params),
                                 ctypes.cast(split, ctypes.c_void_p) if split is not None else None,
                                 ctypes.cast(ph, ctypes.c_void_p), len(fit_phases), _ptr(ws),
                                 ws.numel(), _stream(stream))
    else:
        rc = lib().emdq_batch(ctypes.cast(arr, ctypes.c_void_p), count, ctypes.byref(prm),
                              _ptr(warm_params),
                              ctypes.cast(split, ctypes.c_void_p) if split is not None else None,
                              _ptr(ws), ws.numel(), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_batch', rc)
    return results


def emdq_mosaic(q: torch.Tensor, c: torch.Tensor, src: torch.Tensor, grid, alpha: float,
                frame: torch.Tensor, canvas: torch.Tensor, origin, *,
                workspace: torch.Tensor | None = None, stream=None) -> None:
    """Fused BF16 field + warp: blends frame into canvas through the field of (q, c, src)
    on grid=(x0, y0, w, h), without materialising the field."""
    n = c.shape[0]
    _check(q, 'q', torch.float32, (n, 8))
    _check(c, 'c', torch.float32, (n,))
    _check(src, 'src', torch.float32, (n, 2))
    fw, fh, ch, pitch = _frame_args(frame)
    _check(canvas, 'canvas', torch.uint8)
    if canvas.dim() != 3 or canvas.shape[2] != 4:
        raise ValueError('canvas must be [h, w, 4] uint8')
    chh, cw = canvas.shape[:2]
    x0, y0, gw, gh = (int(v) for v in grid)
    ws = _workspace(field_workspace_size(n, gw, gh, BF16), q.device, workspace)
    rc = lib().emdq_mosaic(_ptr(q), _ptr(c), _ptr(src), n, x0, y0, gw, gh, float(alpha),
                           _ptr(frame), fw, fh, ch, pitch, _ptr(canvas), cw, chh, cw * 4,
                           int(origin[0]), int(origin[1]), _ptr(ws), ws.numel(), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_mosaic', rc)


def mosaic_insert_reference(frame: torch.Tensor, canvas: torch.Tensor, origin, stream=None) -> None:
    fw, fh, ch, pitch = _frame_args(frame)
    _check(canvas, 'canvas', torch.uint8)
    chh, cw = canvas.shape[:2]
    rc = lib().mosaic_insert_reference(_ptr(frame), fw, fh, ch, pitch, _ptr(canvas), cw, chh,
                                       cw * 4, int(origin[0]), int(origin[1]), _stream(stream))
    if rc != 0:
        raise EmdqError('mosaic_insert_reference', rc)


# ---------------------------------------------------------------- learned warm start ----
WARMSTART_PARAMS = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'warmstart_mlp.npy')


def mlp_param_count() -> int:
    return lib().emdq_mlp_param_count()


def warm_features(src: torch.Tensor, dst: torch.Tensor, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """[n, 16] warm-start features of n matches."""
    n = src.shape[0]
    _check(src, 'src', torch.float32, (n, 2))
    _check(dst, 'dst', torch.float32, (n, 2))
    if out is None:
        out = torch.empty((n, 16), dtype=torch.float32, device=src.device)
    _check(out, 'out', torch.float32, (n, 16))
    rc = lib().emdq_warm_features(_ptr(src), _ptr(dst), n, _ptr(out), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_warm_features', rc)
    return out


def warm_infer(feat: torch.Tensor, params: torch.Tensor, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """p0 [n] from features [n, 16] and the 5313 network parameters (float32, CUDA)."""
    n = feat.shape[0]
    _check(feat, 'feat', torch.float32, (n, 16))
    _check(params, 'params', torch.float32, (mlp_param_count(),))
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=feat.device)
    rc = lib().emdq_warm_infer(_ptr(feat), n, _ptr(params), _ptr(out), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_warm_infer', rc)
    return out


def mlp_train_step(feat: torch.Tensor, label: torch.Tensor, params: torch.Tensor,
                   adam_m: torch.Tensor | None, adam_v: torch.Tensor | None, step: int,
                   lr: float, grad_out: torch.Tensor | None = None,
                   loss_out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                   stream=None) -> None:
    """One training step of the warm-start network (step 0: gradient and loss only)."""
    b = feat.shape[0]
    _check(feat, 'feat', torch.float32, (b, 16))
    _check(label, 'label', torch.float32, (b,))
    _check(params, 'params', torch.float32, (mlp_param_count(),))
    ws = _workspace(lib().emdq_mlp_train_workspace_size(b), feat.device, workspace)
    rc = lib().emdq_mlp_train_step(_ptr(feat), _ptr(label), b, _ptr(params), _ptr(adam_m),
                                   _ptr(adam_v), int(step), float(lr), _ptr(grad_out),
                                   _ptr(loss_out), _ptr(ws), ws.numel(), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_mlp_train_step', rc)


def warm_start(problems, params: torch.Tensor, outs: list | None = None, stream=None) -> list:
    """p0 of several problems [(src, dst), ...] in one launch (features + network)."""
    count = len(problems)
    P = ctypes.c_void_p * max(1, count)
    srcs, dsts, p0s = P(), P(), P()
    ns = (ctypes.c_int * max(1, count))()
    out = []
    for b, (src, dst) in enumerate(problems):
        n = src.shape[0]
        _check(src, 'src', torch.float32, (n, 2))
        _check(dst, 'dst', torch.float32, (n, 2))
        o = outs[b] if outs is not None else torch.empty(n, dtype=torch.float32, device=src.device)
        srcs[b], dsts[b], p0s[b], ns[b] = src.data_ptr(), dst.data_ptr(), o.data_ptr(), n
        out.append(o)
    _check(params, 'params', torch.float32, (mlp_param_count(),))
    rc = lib().emdq_warm_start(ctypes.cast(srcs, ctypes.c_void_p), ctypes.cast(dsts, ctypes.c_void_p),
                               ctypes.cast(ns, ctypes.c_void_p), ctypes.cast(p0s, ctypes.c_void_p),
                               count, _ptr(params), _stream(stream))
    if rc != 0:
        raise EmdqError('emdq_warm_start', rc)
    return out


def load_warmstart_params(device='cuda') -> torch.Tensor:
    """The trained warm-start parameters shipped with the package."""
    import numpy as np
    w = np.load(WARMSTART_PARAMS).astype(np.float32)
    if w.shape != (mlp_param_count(),):
        raise ValueError(f'{WARMSTART_PARAMS}: expected {mlp_param_count()} parameters')
    return torch.from_numpy(w).to(device)


def warm_start_p0(src: torch.Tensor, dst: torch.Tensor, params: torch.Tensor, *,
                  feat: torch.Tensor | None = None, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """p0 for emdq_fit: nearest-neighbour features, then the network."""
    feat = warm_features(src, dst, out=feat, stream=stream)
    return warm_infer(feat, params, out=out, stream=stream)
