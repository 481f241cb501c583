"""The input generators (no method arithmetic): the mixed-size batch recipe and the
sequence workloads have the sizes, counts and rates they are stated to have."""
import numpy as np
import pytest

from synth import MIXED_SIZES, WORKLOADS, make_matches, mixed_pairs, workload


def test_mixed_pairs_recipe():
    pairs = mixed_pairs(3, 64)
    assert len(pairs) == 64
    sizes = {(p['scene'].w, p['scene'].h) for p in pairs}
    assert sizes <= set(MIXED_SIZES) and len(sizes) == len(MIXED_SIZES)
    ns = np.array([p['n'] for p in pairs])
    assert ns.min() >= 100 and ns.max() <= 3000 and ns.std() > 400
    for p in pairs:
        assert p['src'].shape == (p['n'], 2) and p['dst'].shape == (p['n'], 2)
        assert 0.10 <= p['outliers'] <= 0.40
        frac = 1.0 - p['inlier'].mean()
        assert abs(frac - p['outliers']) <= 1.5 / p['n'] + 1e-9
        w, h = p['scene'].w, p['scene'].h
        assert (p['src'][:, 0] >= 0).all() and (p['src'][:, 0] <= w - 1).all()
        assert (p['src'][:, 1] >= 0).all() and (p['src'][:, 1] <= h - 1).all()


def test_mixed_pairs_are_seeded():
    a, b = mixed_pairs(5, 4), mixed_pairs(5, 4)
    for x, y in zip(a, b):
        assert np.array_equal(x['src'], y['src']) and np.array_equal(x['dst'], y['dst'])
    c = mixed_pairs(6, 4)
    assert not np.array_equal(a[0]['src'][:10], c[0]['src'][:10])


def test_sequence_workload_shape():
    sc, cfg = workload('seq1280', seed=0)
    assert (sc.w, sc.h, sc.channels) == (1280, 1024, 3) and cfg['frames'] == 100
    s, d, inl = make_matches(sc, 5, cfg['n'], cfg['outliers'], cfg['noise'])
    assert s.shape == (1000, 2) and abs((1 - inl.mean()) - 0.3) < 0.01
    assert set(WORKLOADS) >= {'pair640', 'seq1280', 'warm2000'}


def test_full_sequence_pan_revisits_the_start():
    """The 1920x1080 sequence pans 6 px/frame out for 200 frames and back: frame 400 sees
    the reference view again (up to the drifting bumps), frame 200 is 1200 px away."""
    import math
    import torch
    from synth import gt_forward, make_scene, pan_frames
    sc, cfg = workload('seq1920')
    assert (sc.w, sc.h, cfg['n'], cfg['frames'], cfg['canvas'], cfg['batch']) == \
        (1920, 1080, 5000, 500, (8192, 8192), 8)
    assert math.hypot(*sc.pan) == pytest.approx(6.0)
    assert [pan_frames(sc, t) for t in (0, 1, 200, 201, 399, 400, 450)] == [0, 1, 200, 199, 1, 0, 50]
    still = make_scene(0, 1920, 1080, 3, drift=0.0, pan=sc.pan, pan_turn=sc.pan_turn)
    x = torch.tensor([[10.0, 20.0], [1500.0, 900.0]], dtype=torch.float64)
    assert torch.allclose(gt_forward(still, x, 400), gt_forward(still, x, 0), atol=1e-9)
    shift = gt_forward(still, x, 200) - gt_forward(still, x, 0)
    assert torch.allclose(shift.norm(dim=1), torch.full((2,), 1200.0, dtype=torch.float64))


def test_frame_to_frame_matches():
    """make_pair_matches: inliers sit at the ground-truth positions of their reference points in
    both frames (frame 0 being the reference itself), up to the stated noise in the second."""
    import torch
    from synth import gt_forward, make_pair_matches
    sc, cfg = workload('seq1280', seed=3)
    for t0, t1 in ((0, 1), (4, 5)):
        s, d, inl, x = make_pair_matches(sc, t0, t1, 500, 0.3, 1.0)
        assert s.shape == d.shape == (500, 2) and inl.sum() == 350
        p0 = x[inl] if t0 == 0 else gt_forward(sc, torch.from_numpy(x[inl]), t0).numpy()
        np.testing.assert_allclose(s[inl], p0, atol=1e-3)
        r = d[inl] - gt_forward(sc, torch.from_numpy(x[inl]), t1).numpy()
        assert 0.8 < r.std() < 1.2
        assert np.isnan(x[~inl]).all()
