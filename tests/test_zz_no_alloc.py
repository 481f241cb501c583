"""emdq_fit_noalloc: the allocation-free fit, called through the C ABI, must give what
emdq_fit gives, call after call.

Callers that cannot allocate device memory while running (a real-time video loop where an
allocation could stall the device, a plug-in whose host owns every allocation, a service
with memory fixed at start-up) use this entry point; its scratch is a fixed array inside
the library that every call reuses.  Two calls in a row on different inputs (and
different sizes) check that nothing left in that array by the first call leaks into the
second.
"""
import ctypes

import numpy as np
import pytest
import torch

from synth import make_matches, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    L = pkg.lib()
    P, I = ctypes.c_void_p, ctypes.c_int
    L.emdq_fit_noalloc.restype = I
    L.emdq_fit_noalloc.argtypes = [P, P, I, I, I, ctypes.POINTER(pkg._Params), P, P, P, P, P, P]
    return pkg


def _noalloc_fit(pkg, src, dst, w, h):
    n = src.shape[0]
    q = torch.full((n, 8), float('nan'), device='cuda')
    c = torch.full((n,), float('nan'), device='cuda')
    p = torch.full((n,), float('nan'), device='cuda')
    info = torch.zeros(4, dtype=torch.int32, device='cuda')
    prm = pkg._Params(0.0, 20, 1e-3, 0.25, (ctypes.c_int * 4)())
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = pkg.lib().emdq_fit_noalloc(ptr(src), ptr(dst), n, w, h, ctypes.byref(prm), None, ptr(q),
                                    ptr(c), ptr(p), ptr(info),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, q, c, p, info


def _case(name, seed):
    sc, cfg = workload(name, seed=seed)
    src, dst, _ = make_matches(sc, 1, cfg['n'], cfg['outliers'], cfg['noise'])
    return sc, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()


def test_noalloc_fit_matches_fit_on_two_calls_in_a_row(emdq):
    cases = [_case('seq1280', 11), _case('pair640', 12)]      # N = 1000, then N = 200
    results = []
    for sc, src, dst in cases:                                 # two calls in a row
        rc, q, c, p, info = _noalloc_fit(emdq, src, dst, sc.w, sc.h)
        assert rc == 0, emdq.STATUS.get(rc, rc)
        torch.cuda.synchronize()
        results.append((q.clone(), c.clone(), p.clone(), emdq.read_fit_info(info)))
    for (sc, src, dst), (q, c, p, info) in zip(cases, results):
        ref = emdq.emdq_fit(src, dst, sc.w, sc.h)
        rinfo = emdq.read_fit_info(ref['info'])
        assert info['status_name'] == rinfo['status_name'] == 'OK'
        assert info['iters'] == rinfo['iters']
        # the fit tolerances of the parity tests: posteriors 1e-4, warp rows 2e-3 px
        assert torch.isfinite(q).all() and torch.isfinite(p).all()
        assert (p - ref['p']).abs().max().item() <= 1e-4
        assert ((c > 0) == (ref['c'] > 0)).all()
        x = src.double()
        dq = (q.double() - ref['q'].double()).abs()
        lever = 2.0 * float(x.abs().max()) + 2.0
        assert (dq[:, :4].max().item() * lever) <= 2e-3
        assert (dq[:, 4].max().item() * lever) <= 2e-3
        assert info['sigma2'] == pytest.approx(rinfo['sigma2'], rel=1e-5)


def test_noalloc_calls_allocate_no_device_memory(emdq):
    """After a first call (which looks up the array's address and loads the kernels), further
    calls change neither what torch has allocated nor the device's free memory: the outputs
    are the caller's, the scratch is the library's fixed array."""
    sc, src, dst = _case('seq1280', 13)
    rc, q, c, p, info = _noalloc_fit(emdq, src, dst, sc.w, sc.h)   # warm-up call
    assert rc == 0
    torch.cuda.synchronize()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    prm = emdq._Params(0.0, 20, 1e-3, 0.25, (ctypes.c_int * 4)())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch_before = torch.cuda.memory_allocated()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rc = emdq.lib().emdq_fit_noalloc(ptr(src), ptr(dst), src.shape[0], sc.w, sc.h,
                                         ctypes.byref(prm), None, ptr(q), ptr(c), ptr(p),
                                         ptr(info), stream)
        assert rc == 0
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == torch_before
    assert free_after == free_before
    assert emdq.read_fit_info(info)['status_name'] == 'OK'


def test_noalloc_rejects_sizes_beyond_its_array(emdq):
    n = emdq.lib().emdq_fit_max_n() + 1
    src = torch.zeros((n, 2), device='cuda')
    rc, *_ = _noalloc_fit(emdq, src, src.clone(), 640, 480)
    assert emdq.STATUS[rc] == 'ENOTSUP'
