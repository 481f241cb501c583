"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, 'include', '*.h')):
        src = open(h).read()
        src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
        for m in re.finditer(r'^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(', src, flags=re.M):
            name = m.group(1)
            if name not in ('if', 'sizeof'):
                names.append(name)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ('emdq_fit', 'emdq_field', 'mosaic_warp', 'emdq_fit_workspace_size',
                 'emdq_field_workspace_size'):
        assert must in names


@pytest.fixture(scope='module')
def libemdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return ctypes.CDLL(pkg._LIB_PATH)


def test_library_exports_every_declared_symbol(libemdq):
    for name in declared_functions():
        assert hasattr(libemdq, name), name


def test_library_is_built_for_sm_103a(libemdq):
    import paper_2103_07414_gb300 as pkg
    out = subprocess.run(['cuobjdump', '--list-elf', pkg._LIB_PATH], capture_output=True,
                         text=True)
    if out.returncode != 0:
        pytest.skip('cuobjdump unavailable')
    assert 'sm_103a' in out.stdout


def test_host_only_entry_points(libemdq):
    """Calls that need no GPU: parameters, sizes, status strings, argument checks."""
    import paper_2103_07414_gb300 as pkg
    L = pkg.lib()
    assert L.emdq_abi_version() == 1
    a = L.emdq_alpha_for_frame(480, 270)
    assert abs(a - 2e-4) < 1e-10
    prm = pkg._Params()
    L.emdq_default_params(ctypes.byref(prm))
    assert (prm.max_iters, round(prm.tol_p, 6), prm.sigma2_floor) == (20, 0.001, 0.25)
    assert L.emdq_fit_max_n() >= 5000
    assert L.emdq_fit_workspace_size(1000) >= 4000
    assert L.emdq_status_string(3) == b'EM iteration cap reached (outputs valid)'
    # argument errors are caught on the host before any CUDA call
    rc = L.emdq_fit(None, None, 10, 640, 480, None, None, None, None, None, None, None, 0, None)
    assert rc == 1
    rc = L.emdq_field(None, None, None, 10, 0, 0, 4, 4, ctypes.c_float(1e-3), 0, None, None, 0,
                      None)
    assert rc == 1
    rc = L.mosaic_warp(None, 4, 4, 3, 12, None, 0, 0, 4, 4, None, 8, 8, 32, 0, 0, None)
    assert rc == 1
