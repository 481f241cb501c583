"""The colour bound of the capped running-average blend (Eqs. 23-24 as read), for tests that
compare a GPU canvas with the oracle's (test infrastructure: no arithmetic of the method).

One update is c <- round((w c + v) / (w + 1)).  If two canvases differ by at most D in c before
the update and their two samples by at most e, the two quotients differ by at most
(w D + e) / (w + 1), and two reals that differ by x round to integers at most ceil(x) apart.  So
after the update D' = ceil((w D + e + eta) / (w + 1)), with eta = 1e-3 for the FP32 arithmetic
of the kernel's sample and quotient.  With one field on both sides e is rounding alone, and D
stays at 1 LSB however many frames are blended (w / (w + 1) < 1).  Where the fields differ by
du = u_gpu - u_oracle, a bilinear sample moves by at most |du_x| G_x + |du_y| G_y, with G_x, G_y
the largest differences of horizontally / vertically adjacent frame pixels in the 4 x 4 block
in which both sample positions lie (|du| < 1 px).
"""
import numpy as np

ETA = 1e-3


def lipschitz(frame, ux, uy):
    """Per sample and channel (G_x, G_y): the largest differences of horizontally and
    vertically adjacent pixels of frame [fh, fw, ch] in the block of pixel columns
    floor(ux)-1 .. floor(ux)+2 and rows floor(uy)-1 .. floor(uy)+2 (clipped to the frame)."""
    fh, fw, ch = frame.shape
    x0 = np.floor(ux).astype(np.int64)
    y0 = np.floor(uy).astype(np.int64)
    f = frame.astype(np.int32)
    gx = np.zeros((len(ux), ch), np.int32)
    gy = np.zeros((len(ux), ch), np.int32)
    for dy in range(-1, 3):
        yy = np.clip(y0 + dy, 0, fh - 1)
        yn = np.clip(y0 + dy + 1, 0, fh - 1)
        for dx in range(-1, 3):
            xx = np.clip(x0 + dx, 0, fw - 1)
            xn = np.clip(x0 + dx + 1, 0, fw - 1)
            if dx < 2:
                gx = np.maximum(gx, np.abs(f[yy, xn] - f[yy, xx]))
            if dy < 2:
                gy = np.maximum(gy, np.abs(f[yn, xx] - f[yy, xx]))
    return gx.astype(np.float64), gy.astype(np.float64)


def sample_gap(frame, u_gpu, u_oracle):
    """Per sample and channel: the largest difference of the two bilinear samples of frame at
    u_gpu and u_oracle ([k, 2] each, |u_gpu - u_oracle| < 1)."""
    fh, fw, _ = frame.shape
    du = np.abs(np.asarray(u_gpu, np.float64) - np.asarray(u_oracle, np.float64))
    assert (du < 1.0).all()
    gx, gy = lipschitz(frame, np.clip(u_oracle[:, 0], 0, fw - 1), np.clip(u_oracle[:, 1], 0, fh - 1))
    return du[:, 0:1] * gx + du[:, 1:2] * gy


def carry(D, w_before, e):
    """The bound after one update of pixels with weight w_before ([k]) whose bound was D
    ([k, ch]) and whose samples differ by at most e ([k, ch])."""
    wb = np.asarray(w_before, np.float64)[:, None]
    return np.ceil((wb * D + e + ETA) / (wb + 1.0))
