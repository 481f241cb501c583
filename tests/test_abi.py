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


def test_host_constants_and_node_lattice_against_the_oracle(libemdq, orc):
    """Host-side parts of the node layer, no GPU: the frame-scaled coefficients of Sec. III-G
    (alpha, beta, gamma = 2e-4, 3e-3, 5e-3 over s^2) and the breadth-first node lattice of
    Sec. III-E, the same point set as the oracle's definition (order aside), starting at the
    image centre."""
    import numpy as np
    from scipy.spatial import cKDTree
    import paper_2103_07414_gb300 as pkg
    L = pkg.lib()
    for w, h in ((480, 270), (640, 480), (1280, 1024), (1920, 1080), (333, 917)):
        assert L.emdq_alpha_for_frame(w, h) == pytest.approx(orc.alpha_for_frame(w, h), rel=1e-6)
        assert L.emdq_beta_for_frame(w, h) == pytest.approx(orc.beta_for_frame(w, h), rel=1e-6)
        assert L.emdq_gamma_for_frame(w, h) == pytest.approx(orc.gamma_for_frame(w, h), rel=1e-6)
    for w, h, sp in ((640, 480, 40.0), (1280, 1024, 30.0), (1920, 1080, 55.0), (101, 77, 13.0),
                     (257, 911, 21.5), (5, 3, 100.0)):
        got = pkg.hex_nodes(w, h, sp).numpy().astype(np.float64)
        want = orc.hex_nodes(w, h, sp)
        assert got.shape == want.shape, (w, h, sp)
        np.testing.assert_allclose(got[0], [(w - 1) / 2.0, (h - 1) / 2.0], atol=1e-4)
        d, idx = cKDTree(want).query(got)
        assert d.max() < 1e-3 and len(set(idx.tolist())) == len(want)
    # a short output array receives the first nodes and the full count is returned
    n = L.emdq_hex_nodes(640, 480, 40.0, None, 0)
    buf = (ctypes.c_float * 30)()
    assert L.emdq_hex_nodes(640, 480, 40.0, buf, 10) == n
    np.testing.assert_allclose(np.frombuffer(buf, np.float32)[:20].reshape(10, 2),
                               pkg.hex_nodes(640, 480, 40.0).numpy()[:10])
    assert np.frombuffer(buf, np.float32)[20:].max() == 0.0      # nothing past the capacity
    for bad in ((0, 480, 40.0), (640, -1, 40.0), (640, 480, 0.0), (640, 480, float('nan'))):
        assert L.emdq_hex_nodes(*bad, None, 0) == -1


def test_node_layer_argument_errors_on_the_host(libemdq):
    """The node-layer calls reject bad arguments before any CUDA call (EMDQ_EINVAL = 1)."""
    import paper_2103_07414_gb300 as pkg
    L = pkg.lib()
    f = ctypes.c_float
    assert L.emdq_node_track(None, None, None, 5, None, None, None, 10, f(1e-4), f(1e-3), None,
                             None, None) == 1
    assert L.emdq_node_track(None, None, None, 5, None, None, None, 10, f(-1.0), f(1e-3), None,
                             None, None) == 1
    assert L.emdq_node_merge(None, None, None, None, None, None, 5, f(5e-3), None, None,
                             None) == 1
    assert L.emdq_node_merge(None, None, None, None, None, None, 5, f(0.0), None, None,
                             None) == 1
    assert L.emdq_node_restrict(None, None, 5, None, None, 3, f(3e-3), None, None) == 1
    assert L.emdq_keyframe_distances(None, None, 5, 2, None, None) == 1
    assert L.emdq_feature_uncertainty(None, None, 5, None, None, f(1e-4), f(3e-3), None, None,
                                      None) == 1
    assert L.emdq_node_init(None, None, 5, None, 3, f(1e-4), None, None) == 1
    assert L.emdq_uncertainty(None, None, 5, 0, 0, 4, 4, f(3e-3), None, None) == 1
    assert L.emdq_arap_smooth(None, None, None, 5, f(1e-4), 5, None, None, 0, None) == 1


def test_noalloc_fit_argument_errors_on_the_host(libemdq):
    """emdq_fit_noalloc reports emdq_fit's argument errors first (EMDQ_EINVAL = 1 for a negative
    n or a null pointer, whatever n is) and EMDQ_ENOTSUP (7) only for a valid call with more
    matches than its fixed array holds; all before any CUDA call."""
    import paper_2103_07414_gb300 as pkg
    L = pkg.lib()
    P, I = ctypes.c_void_p, ctypes.c_int
    L.emdq_fit_noalloc.restype = I
    L.emdq_fit_noalloc.argtypes = [P, P, I, I, I, ctypes.POINTER(pkg._Params), P, P, P, P, P, P]
    big = L.emdq_fit_max_n() + 1
    fake = ctypes.c_void_p(1 << 20)           # aligned and never dereferenced: rejected first
    assert L.emdq_fit_noalloc(None, None, -100, 640, 480, None, None, None, None, None, None, None) == 1
    assert L.emdq_fit_noalloc(fake, fake, -100, 640, 480, None, None, fake, fake, None, fake, None) == 1
    assert L.emdq_fit_noalloc(None, None, big, 640, 480, None, None, None, None, None, None, None) == 1
    assert L.emdq_fit_noalloc(fake, fake, big, 640, 0, None, None, fake, fake, None, fake, None) == 1
    assert L.emdq_fit_noalloc(fake, fake, big, 640, 480, None, None, fake, fake, None, fake, None) == 7


def test_mosaic_batch_argument_errors_on_the_host(libemdq):
    """emdq_mosaic_batch rejects bad groups before any CUDA call: a null or empty problem list,
    a bad frame or canvas description (EMDQ_EINVAL = 1), more than 16 frames or a tile height
    other than 16/24/32/40 or a frame of 2^31 bytes or more (EMDQ_ENOTSUP = 7; mosaic_warp
    too), an empty window or one outside the canvas (1),
    and a workspace smaller than its size query or not 256-byte aligned (EMDQ_EWORKSPACE = 6)."""
    import paper_2103_07414_gb300 as pkg
    L = pkg.lib()
    fake = 1 << 20                            # aligned and never dereferenced
    def group(count, grid=(0, 0, 64, 48), n=100):
        arr = (pkg._MosaicProblem * count)()
        for b in range(count):
            arr[b] = pkg._MosaicProblem(fake, fake, fake, n, *grid, 1e-3, fake)
        return ctypes.cast(arr, ctypes.c_void_p)
    cv = ctypes.c_void_p(fake)
    args = lambda g, k: (g, k, 640, 480, 3, 1920, cv, 1000, 800, 4000, 10, 10)
    ws = ctypes.c_void_p(1 << 24)
    size = L.emdq_mosaic_batch_workspace_size(group(2), 2)
    assert size > 1024
    assert L.emdq_mosaic_batch_workspace_size(group(17), 17) == 0
    assert L.emdq_mosaic_batch(None, 1, *args(None, 1)[2:], ws, size, None) == 1
    assert L.emdq_mosaic_batch(*args(group(1), 0), ws, size, None) == 1
    assert L.emdq_mosaic_batch(group(1), 1, 640, 480, 2, 1920, cv, 1000, 800, 4000, 10, 10, ws, size, None) == 1
    assert L.emdq_mosaic_batch(group(1), 1, 640, 480, 3, 1000, cv, 1000, 800, 4000, 10, 10, ws, size, None) == 1
    assert L.emdq_mosaic_batch(group(1), 1, 640, 480, 3, 1920, cv, 1000, 800, 3999, 10, 10, ws, size, None) == 1
    assert L.emdq_mosaic_batch(*args(group(17), 17), ws, size, None) == 7
    assert L.emdq_mosaic_batch_ex(*args(group(2), 2), 48, ws, size, None) == 7
    assert L.emdq_mosaic_batch(*args(group(1, grid=(0, 0, 0, 48)), 1), ws, size, None) == 1
    assert L.emdq_mosaic_batch(*args(group(1, grid=(985, 0, 10, 10)), 1), ws, size, None) == 1
    assert L.emdq_mosaic_batch(*args(group(1, grid=(-11, 0, 10, 10)), 1), ws, size, None) == 1
    assert L.emdq_mosaic_batch(group(1), 1, 640, 1024, 3, 1 << 21, cv, 1000, 800, 4000, 10, 10, ws, size, None) == 7
    assert L.mosaic_warp(fake, 640, 1024, 3, 1 << 21, fake, 0, 0, 4, 4, fake, 8, 8, 32, 0, 0, None) == 7
    assert L.emdq_mosaic_batch(*args(group(2), 2), ws, size - 1, None) == 6
    assert L.emdq_mosaic_batch(*args(group(2), 2), ctypes.c_void_p(fake + 16), size, None) == 6


def test_mosaic_pairs_argument_errors_on_the_host(libemdq):
    """emdq_mosaic_pairs rejects bad pair lists before any CUDA call: no pairs, channels other
    than 1 or 3, a bad frame or canvas description or a window outside its canvas (EMDQ_EINVAL
    = 1), two pairs whose windows cover overlapping canvas rows (1, whether they share the
    canvas pointer or not), more than 16 pairs or a frame of 2^31 bytes or more (EMDQ_ENOTSUP =
    7), and a workspace smaller than its size query or not 256-byte aligned (EMDQ_EWORKSPACE =
    6).  Pairs on disjoint canvases pass the checks."""
    import paper_2103_07414_gb300 as pkg
    L = pkg.lib()
    fake = 1 << 20                            # aligned and never dereferenced
    def pairs(specs):
        arr = (pkg._MosaicPair * len(specs))()
        for b, sp in enumerate(specs):
            d = dict(grid=(0, 0, 64, 48), canvas=fake + b * (1 << 24), cw=1000, ch=800, pitch=4000,
                     origin=(10, 10), fw=640, fh=480, fpitch=1920, n=100)
            d.update(sp)
            arr[b] = pkg._MosaicPair(fake, fake, fake, d['n'], *d['grid'], 1e-3, fake, d['fw'], d['fh'],
                                     d['fpitch'], d['canvas'], d['cw'], d['ch'], d['pitch'], *d['origin'])
        return ctypes.cast(arr, ctypes.c_void_p), len(specs)
    ws = ctypes.c_void_p(1 << 40)
    two = pairs([{}, {}])
    size = L.emdq_mosaic_pairs_workspace_size(*two)
    assert size > 1024
    assert L.emdq_mosaic_pairs_workspace_size(*pairs([{}] * 17)) == 0
    assert L.emdq_mosaic_pairs(None, 1, 3, ws, size, None) == 1
    assert L.emdq_mosaic_pairs(two[0], 0, 3, ws, size, None) == 1
    assert L.emdq_mosaic_pairs(*two, 2, ws, size, None) == 1
    assert L.emdq_mosaic_pairs(*pairs([{}, {'fpitch': 1000}]), 3, ws, size, None) == 1
    assert L.emdq_mosaic_pairs(*pairs([{}, {'pitch': 3999}]), 3, ws, size, None) == 1
    assert L.emdq_mosaic_pairs(*pairs([{}, {'grid': (985, 0, 10, 10)}]), 3, ws, size, None) == 1
    assert L.emdq_mosaic_pairs(*pairs([{}, {'grid': (0, 0, 0, 48)}]), 3, ws, size, None) == 1
    # the same canvas: overlapping windows, and windows side by side in the same rows
    assert L.emdq_mosaic_pairs(*pairs([{'canvas': fake}, {'canvas': fake, 'grid': (30, 20, 64, 48)}]),
                               3, ws, size, None) == 1
    assert L.emdq_mosaic_pairs(*pairs([{'canvas': fake}, {'canvas': fake, 'grid': (200, 0, 64, 48)}]),
                               3, ws, size, None) == 1
    # a second canvas view that starts inside the first one's rows
    assert L.emdq_mosaic_pairs(*pairs([{'canvas': fake}, {'canvas': fake + 4000 * 20}]), 3, ws, size,
                               None) == 1
    assert L.emdq_mosaic_pairs(*pairs([{}] * 17), 3, ws, size, None) == 7
    assert L.emdq_mosaic_pairs(*pairs([{}, {'fh': 1024, 'fpitch': 1 << 21}]), 3, ws, size, None) == 7
    assert L.emdq_mosaic_pairs(*two, 3, ws, size - 1, None) == 6
    assert L.emdq_mosaic_pairs(*two, 3, ctypes.c_void_p((1 << 40) + 16), size, None) == 6
    # the same canvas, windows in disjoint rows: accepted by the checks (the workspace is then
    # refused, so that nothing is launched)
    assert L.emdq_mosaic_pairs(*pairs([{'canvas': fake}, {'canvas': fake, 'grid': (0, 100, 64, 48)}]),
                               3, ws, size - 1, None) == 6


def test_fit_batch_phases_argument_errors_on_the_host(libemdq):
    """emdq_fit_batch_phases rejects, before any CUDA call (EMDQ_EINVAL = 1): no phases, more
    than 16, counts that do not increase or are below 1, and a problem without p_out (a later
    phase starts from it)."""
    import paper_2103_07414_gb300 as pkg
    L = pkg.lib()
    fake = 1 << 20
    arr = (pkg._Problem * 2)()
    for b in range(2):
        arr[b] = pkg._Problem(fake, fake, 100, 640, 480, None, fake, fake, fake, fake)
    probs = ctypes.cast(arr, ctypes.c_void_p)
    ws = ctypes.c_void_p(1 << 24)
    def call(phases, pr=probs):
        ph = (ctypes.c_int * max(1, len(phases)))(*phases)
        return L.emdq_fit_batch_phases(pr, 2, None, ctypes.cast(ph, ctypes.c_void_p), len(phases),
                                       ws, 1 << 30, None)
    assert call([]) == 1
    assert call(list(range(1, 18))) == 1
    assert call([5, 5]) == 1
    assert call([6, 4]) == 1
    assert call([0, 4]) == 1
    arr[1] = pkg._Problem(fake, fake, 100, 640, 480, None, fake, fake, None, fake)
    assert call([6, 10]) == 1


def test_warm_start_training_initialisation_on_the_host():
    """The package's training starts from He-normal weights in the kernels' packed layout:
    5313 parameters, zero biases, deterministic per seed (no GPU needed)."""
    import torch
    from paper_2103_07414_gb300.training import init_params
    p = init_params(3, device='cpu')
    q = init_params(3, device='cpu')
    assert p.shape == (16 * 64 + 64 + 64 * 64 + 64 + 64 + 1,) and p.dtype == torch.float32
    assert torch.equal(p, q) and not torch.equal(p, init_params(4, device='cpu'))
    W1, b1 = p[:1024], p[1024:1088]
    W2, b2 = p[1088:5184], p[5184:5248]
    assert float(b1.abs().max()) == 0.0 and float(b2.abs().max()) == 0.0 and float(p[-1]) == 0.0
    assert abs(float(W1.std()) - (2 / 16) ** 0.5) < 0.05 and abs(float(W2.std()) - (2 / 64) ** 0.5) < 0.02
