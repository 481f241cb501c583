"""GPU parity: emdq_field (C ABI) against the oracle's FP64 field (Eqs. 2-4)."""
import math

import numpy as np
import pytest
import torch

from gpu_cases import fitted_case, random_rows

pytestmark = pytest.mark.gpu

# Field tolerances vs the FP64 oracle, px (maximum over every compared pixel).
TOL = {0: 1e-3, 1: 0.05}


@pytest.fixture(scope='module')
def emdq():
    import paper_2103_07414_gb300 as pkg
    pkg.build()
    return pkg


def _gpu_field(emdq, q8, c, src, grid, alpha, prec):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    d = emdq.emdq_field(t(q8), t(c), t(src), grid, alpha, precision=prec)
    torch.cuda.synchronize()
    return d.cpu().numpy().astype(np.float64)


def _oracle_inputs(q8, c, src):
    # the oracle sees exactly the float32 values the GPU reads
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    return f(q8), f(c), f(src)


PRECISIONS = [0, 1]


@pytest.mark.parametrize('prec', PRECISIONS, ids=['fp32', 'bf16'])
def test_field_parity_fitted_pair(emdq, orc, prec):
    sc, cfg, src, dst, inl, r = fitted_case(orc, 'pair640', seed=0)
    alpha = orc.alpha_for_frame(sc.w, sc.h)
    grid = (-7, -5, 333, 141)                     # ragged in both directions
    q8, c, s = _oracle_inputs(r['q8'], r['c'], src)
    want = orc.field(q8, c, s, grid, alpha)
    got = _gpu_field(emdq, r['q8'], r['c'], src, grid, np.float32(alpha), prec)
    err = np.abs(got - want).max()
    print(f'prec {prec}: max field error {err:.3e} px')
    assert err <= TOL[prec]


def test_field_tiny_brute_force_8d_dq(emdq, orc):
    """N = 3..8 on a 16x16 grid, the FP32 path against an independent 8-D dual-quaternion
    blend (Kavan) in float64, not against the oracle.  (The BF16 path's worst-case operand
    rounding on rows this far apart exceeds its tolerance; it is held to the oracle on the
    workloads' transforms instead.)"""
    from dq8 import axis_angle, dq_from_rotation_translation, dqb_point
    rng = np.random.default_rng(16)
    alpha = np.float32(0.01)
    for trial in range(4):
        n = int(rng.integers(3, 9))
        src = rng.uniform(0, 16, (n, 2)).astype(np.float32)
        ths = rng.uniform(-0.5, 0.5, n)
        ts = rng.uniform(-20, 20, (n, 2))
        ss = rng.uniform(0.8, 1.25, n)
        c = rng.uniform(0.0, 1.0, n).astype(np.float32)
        c[0] = 1.0
        q8 = np.stack([[*orc.dq_from_rt(ths[i], ts[i, 0], ts[i, 1]), ss[i], 1.0, 0.0, 0.0]
                       for i in range(n)])
        reals, duals = zip(*[dq_from_rotation_translation(axis_angle([0, 0, 1], ths[i]),
                                                          [ts[i, 0], ts[i, 1], 0.0])
                             for i in range(n)])
        reals, duals = np.array(reals), np.array(duals)
        got = _gpu_field(emdq, q8, c, src, (0, 0, 16, 16), alpha, 0)
        s64, c64 = src.astype(np.float64), c.astype(np.float64)
        err = 0.0
        for y in range(16):
            for x in range(16):
                w = c64 * np.exp(-float(alpha) * ((s64 - [x, y]) ** 2).sum(1))
                want = dqb_point(w, ss, reals, duals, (x, y))
                err = max(err, float(np.abs(got[y, x] - (want[:2] - [x, y])).max()))
        print(f'n={n}: max error against the 8-D DQ blend {err:.2e} px')
        assert err <= TOL[0]


@pytest.mark.parametrize('prec', PRECISIONS, ids=['fp32', 'bf16'])
def test_field_identical_transforms(emdq, orc, prec):
    rng = np.random.default_rng(2)
    n = 300
    src = rng.uniform(0, 1279, (n, 2))
    q = orc.dq_from_rt(math.radians(5), 12.0, -7.0)
    q8 = np.tile([q[0], q[1], q[2], q[3], 1.05, 1, 0, 0], (n, 1))
    c = rng.uniform(0.5, 1.0, n)
    grid = (0, 0, 1280, 64)
    alpha = orc.alpha_for_frame(1280, 1024)
    got = _gpu_field(emdq, q8, c, src, grid, np.float32(alpha), prec)
    want = orc.field(*_oracle_inputs(q8, c, src), grid, alpha)
    assert np.abs(got - want).max() <= TOL[prec]


@pytest.mark.parametrize('prec', PRECISIONS, ids=['fp32', 'bf16'])
def test_field_no_weight_gives_nan(emdq, prec):
    n = 40
    t = lambda a: torch.tensor(a, dtype=torch.float32, device='cuda')
    q8 = t(np.tile([1, 0, 0, 0, 1, 1, 0, 0], (n, 1)))
    d = emdq.emdq_field(q8, torch.zeros(n, device='cuda'), torch.rand(n, 2, device='cuda') * 10,
                        (0, 0, 20, 3), 1e-3, precision=prec)
    assert torch.isnan(d).all()


@pytest.mark.parametrize('prec', PRECISIONS, ids=['fp32', 'bf16'])
def test_field_full_size_sampled(emdq, orc, prec):
    """1280x1024 frame, N=1000, the benchmark's launch; compare 4096 sampled pixels."""
    rng = np.random.default_rng(3)
    src, q8 = random_rows(rng, 1000, 1280, 1024)
    c = np.where(rng.uniform(0, 1, 1000) < 0.7, rng.uniform(0.5, 1, 1000), 0.0)
    grid = (-30, -40, 1340, 1100)
    alpha = orc.alpha_for_frame(1280, 1024)
    got = _gpu_field(emdq, q8, c, src, grid, np.float32(alpha), prec)
    iy = rng.integers(0, grid[3], 4096)
    ix = rng.integers(0, grid[2], 4096)
    pts = np.stack([grid[0] + ix, grid[1] + iy], 1).astype(np.float64)
    want = orc.field_points(*_oracle_inputs(q8, c, src), pts, alpha)
    err = np.abs(got[iy, ix] - want).max()
    print(f'prec {prec}: full-size sampled max error {err:.3e} px')
    assert err <= TOL[prec]


def test_field_bad_arguments(emdq):
    q8 = torch.zeros((4, 8), device='cuda')
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_field(q8, torch.ones(4, device='cuda'), torch.zeros(4, 2, device='cuda'),
                        (0, 0, 4, 4), -1.0, precision=0)


@pytest.mark.parametrize('prec', PRECISIONS, ids=['fp32', 'bf16'])
@pytest.mark.parametrize('n', [3, 65, 129])
def test_field_small_and_ragged_match_counts(emdq, orc, prec, n):
    """Match counts that leave most of a 64-match slice as padding; one-tile grids."""
    rng = np.random.default_rng(100 + n)
    src, q8 = random_rows(rng, n, 640, 480)
    c = rng.uniform(0.3, 1.0, n)
    alpha = orc.alpha_for_frame(640, 480)
    for grid in [(5, 7, 17, 9), (-3, 100, 128, 32), (0, 0, 129, 33)]:
        got = _gpu_field(emdq, q8, c, src, grid, np.float32(alpha), prec)
        want = orc.field(*_oracle_inputs(q8, c, src), grid, alpha)
        assert np.abs(got - want).max() <= TOL[prec], (grid, np.abs(got - want).max())


@pytest.mark.parametrize('prec', PRECISIONS, ids=['fp32', 'bf16'])
@pytest.mark.parametrize('m', [1, 63, 64, 65, 128, 129])
def test_field_sparse_weights(emdq, orc, prec, m):
    """Only m of 300 matches carry weight (scattered, so the nonzero columns the tensor path
    keeps land on either side of its 64-match slices); the zero-weight ones must not count."""
    rng = np.random.default_rng(200 + m)
    n = 300
    src, q8 = random_rows(rng, n, 640, 480)
    c = np.zeros(n)
    c[rng.choice(n, m, replace=False)] = rng.uniform(0.5, 1.0, m)
    alpha = orc.alpha_for_frame(640, 480)
    grid = (-3, 11, 200, 45)
    got = _gpu_field(emdq, q8, c, src, grid, np.float32(alpha), prec)
    want = orc.field(*_oracle_inputs(q8, c, src), grid, alpha)
    ok = np.isfinite(want)
    assert np.array_equal(np.isfinite(got), ok)
    assert np.abs(got[ok] - want[ok]).max() <= TOL[prec]


@pytest.mark.parametrize('prec', PRECISIONS, ids=['fp32', 'bf16'])
def test_field_many_matches_sampled(emdq, orc, prec):
    """n = 9000 (beyond the tensor path's 8192-match column compaction: all columns are
    kept), 30 % zero weights; 2048 sampled pixels."""
    rng = np.random.default_rng(9000)
    n = 9000
    src, q8 = random_rows(rng, n, 1280, 1024)
    c = np.where(rng.uniform(0, 1, n) < 0.7, rng.uniform(0.5, 1, n), 0.0)
    grid = (0, 0, 1280, 256)
    alpha = orc.alpha_for_frame(1280, 1024)
    got = _gpu_field(emdq, q8, c, src, grid, np.float32(alpha), prec)
    iy = rng.integers(0, grid[3], 2048)
    ix = rng.integers(0, grid[2], 2048)
    pts = np.stack([grid[0] + ix, grid[1] + iy], 1).astype(np.float64)
    want = orc.field_points(*_oracle_inputs(q8, c, src), pts, alpha)
    err = np.abs(got[iy, ix] - want).max()
    print(f'prec {prec}: n=9000 sampled max error {err:.3e} px')
    assert err <= TOL[prec]


def _field_case(rng, n, w, h, zero_frac=0.3):
    src, q8 = random_rows(rng, n, w, h)
    c = np.where(rng.uniform(0, 1, n) < 1 - zero_frac, rng.uniform(0.5, 1, n), 0.0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    return t(q8), t(c), t(src), (q8, c, src)


def test_field_batch_equals_single_calls(emdq):
    """One operand launch and one persistent GEMM over several fields give each field
    bit for bit what its own emdq_field (BF16) call gives."""
    rng = np.random.default_rng(77)
    specs = [(1000, 1280, 1024, (-30, -40, 1343, 1083)), (137, 640, 480, (5, 7, 17, 9)),
             (2500, 1920, 1080, (-12, 3, 1999, 700)), (64, 640, 480, (0, 0, 129, 33)),
             (900, 1280, 720, (100, -20, 640, 300))]
    probs = []
    for n, w, h, grid in specs:
        q, c, s, _ = _field_case(rng, n, w, h)
        probs.append((q, c, s, grid, np.float32(emdq.alpha_for_frame(w, h))))
    got = emdq.emdq_field_batch(probs)
    torch.cuda.synchronize()
    for (q, c, s, grid, alpha), g in zip(probs, got):
        want = emdq.emdq_field(q, c, s, grid, alpha, precision=emdq.BF16)
        torch.cuda.synchronize()
        assert torch.equal(torch.isnan(g), torch.isnan(want))
        assert torch.equal(torch.nan_to_num(g), torch.nan_to_num(want))


def test_field_batch_of_16_against_the_oracle(emdq, orc):
    rng = np.random.default_rng(78)
    probs, host = [], []
    for b in range(16):
        w, h = [(640, 480), (1280, 720), (1280, 1024), (1920, 1080)][b % 4]
        n = int(rng.integers(100, 1500))
        q, c, s, hq = _field_case(rng, n, w, h)
        grid = (int(rng.integers(-20, 20)), int(rng.integers(-20, 20)), int(rng.integers(200, 400)),
                int(rng.integers(40, 120)))
        alpha = np.float32(orc.alpha_for_frame(w, h))
        probs.append((q, c, s, grid, alpha))
        host.append((hq, grid, alpha))
    got = emdq.emdq_field_batch(probs)
    torch.cuda.synchronize()
    for g, ((q8, c, s), grid, alpha) in zip(got, host):
        want = orc.field(*_oracle_inputs(q8, c, s), grid, float(alpha))
        assert np.abs(g.cpu().numpy().astype(np.float64) - want).max() <= TOL[1]


def test_field_batch_errors(emdq):
    rng = np.random.default_rng(79)
    q, c, s, _ = _field_case(rng, 50, 640, 480)
    p = (q, c, s, (0, 0, 64, 32), 1e-4)
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_field_batch([p] * 17)
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_field_batch([(q, c, s, (0, 0, 64, 32), -1.0)])
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_field_batch([(q, c, s, (0, 0, 0, 32), 1e-4)])


@pytest.mark.parametrize('tile_rows', [16, 24, 40])
def test_field_batch_every_tile_height_gives_the_same_bits(emdq, tile_rows):
    """The tile height changes only how the GEMM covers the window: every output's
    accumulation over the matches is the same, so the fields are bit for bit those of the
    default tile height, on ragged windows (heights that are no multiple of any tile)."""
    rng = np.random.default_rng(80 + tile_rows)
    specs = [(1000, 1280, 1024, (-30, -40, 1343, 1083)), (137, 640, 480, (5, 7, 17, 9)),
             (2500, 1920, 1080, (-12, 3, 1999, 701)), (64, 640, 480, (0, 0, 129, 33))]
    probs = []
    for n, w, h, grid in specs:
        q, c, s, _ = _field_case(rng, n, w, h)
        probs.append((q, c, s, grid, np.float32(emdq.alpha_for_frame(w, h))))
    ref = emdq.emdq_field_batch(probs, tile_rows=32)
    got = emdq.emdq_field_batch(probs, tile_rows=tile_rows)
    torch.cuda.synchronize()
    for g, r in zip(got, ref):
        assert torch.equal(torch.isnan(g), torch.isnan(r))
        assert torch.equal(torch.nan_to_num(g), torch.nan_to_num(r))


def test_field_batch_autotune_records_its_choice(emdq):
    """The autotuner times every tile height, returns the fastest and records it for the
    batch's size class: emdq_field_batch then uses it (and a bad height is refused)."""
    rng = np.random.default_rng(90)
    probs = []
    for _ in range(3):
        q, c, s, _ = _field_case(rng, 700, 1280, 1024)
        probs.append((q, c, s, (-10, -20, 1300, 1070), np.float32(emdq.alpha_for_frame(1280, 1024))))
    before = emdq.emdq_field_batch(probs, tile_rows=32)
    py, ms = emdq.field_batch_autotune(probs, reps=3)
    print(f'chosen tile height {py}, {ms * 1e3:.1f} us per call')
    assert py in (16, 24, 32, 40) and ms > 0
    assert emdq.field_batch_tile_rows(probs) == py
    after = emdq.emdq_field_batch(probs)
    torch.cuda.synchronize()
    for a, b in zip(after, before):
        assert torch.equal(torch.nan_to_num(a), torch.nan_to_num(b))
    with pytest.raises(emdq.EmdqError):
        emdq.emdq_field_batch(probs, tile_rows=48)
