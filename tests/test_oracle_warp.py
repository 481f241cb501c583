"""Pins of the oracle's gather warp and capped running-average blend (Sec. III-F)."""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden', 'parameters.json')


def _canvas(cw=64, ch=48):
    return np.zeros((ch, cw, 4), np.uint8)


def _const_disp(gw, gh, dx, dy):
    d = np.empty((gh, gw, 2), np.float32)
    d[..., 0], d[..., 1] = dx, dy
    return d


def test_zero_field_copies_the_frame(orc):
    rng = np.random.default_rng(1)
    frame = rng.integers(0, 256, (20, 30, 3), dtype=np.uint8)
    cv = _canvas()
    origin = (10, 12)
    assert orc.warp(frame, _const_disp(30, 20, 0, 0), (0, 0, 30, 20), cv, origin) == 0
    np.testing.assert_array_equal(cv[12:32, 10:40, :3], frame)
    assert (cv[12:32, 10:40, 3] == 1).all()
    assert (cv[:12] == 0).all() and (cv[32:] == 0).all()


def test_integer_translation_shifts_exactly(orc):
    rng = np.random.default_rng(2)
    frame = rng.integers(0, 256, (20, 30), dtype=np.uint8)
    cv = _canvas()
    # canvas pixel p samples the frame at p + (3, -2); the window covers p in [-3..26]x[2..21]
    grid = (-5, 0, 40, 25)
    orc.warp(frame, _const_disp(40, 25, 3.0, -2.0), grid, cv, (8, 10))
    for py in range(0, 25):
        for px in range(-5, 35):
            ux, uy = px + 3, py - 2
            pix = cv[py + 10, px + 8]
            if 0 <= ux <= 29 and 0 <= uy <= 19:
                assert pix[0] == frame[uy, ux] and pix[3] == 1
            else:
                assert pix[3] == 0 and pix[0] == 0


def test_bilinear_is_exact_on_a_linear_ramp(orc):
    ys, xs = np.mgrid[0:16, 0:16]
    frame = (5 * xs + 7 * ys + 10).astype(np.uint8)     # max 190
    rng = np.random.default_rng(3)
    d = rng.uniform(-0.5, 0.5, (8, 8, 2)).astype(np.float32)
    cv = _canvas(32, 32)
    orc.warp(frame, d, (4, 4, 8, 8), cv, (0, 0))
    for y in range(8):
        for x in range(8):
            ux = np.float32(np.float32(4 + x) + d[y, x, 0])
            uy = np.float32(np.float32(4 + y) + d[y, x, 1])
            v = 5 * float(ux) + 7 * float(uy) + 10
            assert cv[4 + y, 4 + x, 0] == np.floor(v + 0.5)


def test_edges_are_inside_and_beyond_is_untouched(orc):
    frame = np.full((10, 10), 200, np.uint8)
    cv = _canvas(16, 16)
    d = np.zeros((1, 4, 2), np.float32)
    d[0, :, 0] = [0.0, -1.001, 7.0, 6.001]               # u_x = 0, -0.001 (out), 9, 9.001 (out)
    orc.warp(frame, d, (0, 0, 4, 1), cv, (0, 0))
    assert list(cv[0, :4, 3]) == [1, 0, 1, 0]
    assert list(cv[0, :4, 0]) == [200, 0, 200, 0]
    # NaN displacement: untouched
    cv2 = _canvas(16, 16)
    orc.warp(frame, np.full((1, 1, 2), np.nan, np.float32), (0, 0, 1, 1), cv2, (0, 0))
    assert (cv2 == 0).all()


def test_running_average_and_the_weight_cap(orc):
    cap = json.load(open(GOLDEN))['merge_weight_cap']['value']
    frame = np.full((4, 4), 77, np.uint8)
    cv = _canvas(8, 8)
    for k in range(cap + 1):
        orc.warp(frame, _const_disp(4, 4, 0, 0), (0, 0, 4, 4), cv, (0, 0))
        assert (cv[:4, :4, 3] == min(k + 1, cap)).all()
        assert (cv[:4, :4, 0] == 77).all()
    # one different frame after saturation moves the value by 1/(cap + 1) of the step
    orc.warp(np.full((4, 4), 77 + 62, np.uint8), _const_disp(4, 4, 0, 0), (0, 0, 4, 4), cv, (0, 0))
    assert (cv[:4, :4, 0] == 79).all() and (cv[:4, :4, 3] == cap).all()


def test_blend_is_order_dependent(orc):
    a = np.full((2, 2), 10, np.uint8)
    b = np.full((2, 2), 101, np.uint8)
    z = _const_disp(2, 2, 0, 0)
    cv1, cv2 = _canvas(2, 2), _canvas(2, 2)
    for f in (a, a, b):
        orc.warp(f, z, (0, 0, 2, 2), cv1, (0, 0))
    for f in (b, a, a):
        orc.warp(f, z, (0, 0, 2, 2), cv2, (0, 0))
    assert cv1[0, 0, 0] == 40          # (2*10 + 101)/3 = 40.33
    assert cv2[0, 0, 0] == 41          # 10 + ... : (55.5 -> 56), (2*56 + 10)/3 = 40.67
    assert cv1[0, 0, 3] == cv2[0, 0, 3] == 3


def test_window_outside_canvas_is_rejected(orc):
    frame = np.zeros((4, 4), np.uint8)
    cv = _canvas(8, 8)
    assert orc.warp(frame, _const_disp(4, 4, 0, 0), (6, 6, 4, 4), cv, (0, 0)) == 1


def test_insert_reference(orc):
    rng = np.random.default_rng(4)
    f = rng.integers(0, 256, (5, 6, 3), dtype=np.uint8)
    cv = _canvas(10, 10)
    assert orc.insert_reference(f, cv, (2, 3)) == 0
    np.testing.assert_array_equal(cv[3:8, 2:8, :3], f)
    assert (cv[3:8, 2:8, 3] == 1).all() and cv[..., 3].sum() == 30


def test_frame_rows_are_read_through_the_pitch(orc):
    """A frame stored inside a wider buffer (rows further apart than w x channels bytes, other
    data between them) warps and inserts exactly as the same frame stored tightly."""
    rng = np.random.default_rng(5)
    buf = rng.integers(0, 256, (20, 41, 3), dtype=np.uint8)     # 11 columns of other data per row
    view = buf[:, :30]
    tight = np.ascontiguousarray(view)
    d = rng.uniform(-3, 3, (24, 36, 2)).astype(np.float32)
    a, b = _canvas(), _canvas()
    orc.warp(view, d, (-3, -2, 36, 24), a, (10, 12))
    orc.warp(tight, d, (-3, -2, 36, 24), b, (10, 12))
    np.testing.assert_array_equal(a, b)
    assert (a[..., 3] > 0).sum() > 400
    a, b = _canvas(), _canvas()
    orc.insert_reference(view, a, (5, 6))
    orc.insert_reference(tight, b, (5, 6))
    np.testing.assert_array_equal(a, b)


def test_rgb_channels_are_sampled_separately(orc):
    """Three channels holding three different linear ramps: bilinear sampling is exact on each."""
    ys, xs = np.mgrid[0:16, 0:16]
    coef = [(5, 7, 10), (3, 2, 40), (9, 1, 5)]                       # maxima 190, 115, 155
    frame = np.stack([a * xs + b * ys + c for a, b, c in coef], -1).astype(np.uint8)
    rng = np.random.default_rng(6)
    d = rng.uniform(-0.5, 0.5, (8, 8, 2)).astype(np.float32)
    cv = _canvas(32, 32)
    orc.warp(frame, d, (4, 4, 8, 8), cv, (0, 0))
    for y in range(8):
        for x in range(8):
            ux = float(np.float32(np.float32(4 + x) + d[y, x, 0]))
            uy = float(np.float32(np.float32(4 + y) + d[y, x, 1]))
            for k, (a, b, c) in enumerate(coef):
                assert cv[4 + y, 4 + x, k] == np.floor(a * ux + b * uy + c + 0.5)


def test_sample_position_is_formed_in_float32(orc):
    """The sample position u = p + d is rounded to FP32 before the coverage test (the kernel's
    precision): 2^-22 past the last column rounds back onto it and is inside."""
    frame = np.full((10, 10), 90, np.uint8)
    cv = _canvas(16, 16)
    d = np.zeros((1, 2, 2), np.float32)
    d[0, :, 0] = 2.0 ** -22                 # p = 8: inside; p = 9: 9 + 2^-22 rounds to 9.0
    orc.warp(frame, d, (8, 0, 2, 1), cv, (0, 0))
    assert list(cv[0, 8:10, 3]) == [1, 1] and list(cv[0, 8:10, 0]) == [90, 90]
