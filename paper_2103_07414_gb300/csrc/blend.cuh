// Per-pixel gather + bilinear sample + capped running-average blend (Sec. III-F,
// Eqs. 23-24 as read), shared by the stand-alone warp kernel and the fused tensor-core
// field epilogue so that both paths compute the same bits.  Split in three steps (tap
// set-up, loads, update) so that a thread handling several pixels can issue all their
// loads before it uses any.
#pragma once

#include "common.cuh"

namespace emdq {

// Where a canvas pixel samples frame t: u = p + d with one FP32 rounding per axis; valid
// iff u lies in [0, fw-1] x [0, fh-1] (a NaN d is invalid); bilinear taps and weights.
struct Tap {
    int r0, r1, c0, c1;     // byte offsets of the two rows and two columns
    float w00, w10, w01, w11;
    bool ok;
};

template <int CH>
__device__ __forceinline__ Tap tap_setup(int fw, int fh, int pitch, float px, float py, float dx,
                                         float dy)
{
    Tap t;
    const float ux = __fadd_rn(px, dx);
    const float uy = __fadd_rn(py, dy);
    t.ok = ux >= 0.f && ux <= static_cast<float>(fw - 1) && uy >= 0.f &&
           uy <= static_cast<float>(fh - 1);
    if (!t.ok) {
        t.r0 = t.r1 = t.c0 = t.c1 = 0;
        t.w00 = t.w10 = t.w01 = t.w11 = 0.f;
        return t;
    }
    const int x0 = static_cast<int>(floorf(ux)), y0 = static_cast<int>(floorf(uy));
    const float fx = ux - static_cast<float>(x0), fy = uy - static_cast<float>(y0);
    const int x1 = min(x0 + 1, fw - 1), y1 = min(y0 + 1, fh - 1);
    t.w00 = (1.f - fx) * (1.f - fy);
    t.w10 = fx * (1.f - fy);
    t.w01 = (1.f - fx) * fy;
    t.w11 = fx * fy;
    t.r0 = y0 * pitch;
    t.r1 = y1 * pitch;
    t.c0 = x0 * CH;
    t.c1 = x1 * CH;
    return t;
}

template <int CH>
__device__ __forceinline__ void tap_sample(const uint8_t *__restrict__ frame, const Tap &t,
                                           float (&v)[CH])
{
    // byte offsets in 32 bits (a frame holds fewer than 2^31 bytes; the entry points check)
    const uint8_t *p00 = frame + static_cast<unsigned>(t.r0 + t.c0);
    const uint8_t *p10 = frame + static_cast<unsigned>(t.r0 + t.c1);
    const uint8_t *p01 = frame + static_cast<unsigned>(t.r1 + t.c0);
    const uint8_t *p11 = frame + static_cast<unsigned>(t.r1 + t.c1);
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        v[k] = t.w00 * __ldg(p00 + k) + t.w10 * __ldg(p10 + k) + t.w01 * __ldg(p01 + k) +
               t.w11 * __ldg(p11 + k);
    }
}

// c <- clamp(floor((w c + v)/(w + 1) + 1/2), 0, 255).  w c + v is exact for integer v and
// the quotient is correctly rounded, so ties land exactly on .5 as in FP64.  The quotient
// a / b comes from the correctly rounded reciprocal y = RN(1/b), taken once per pixel, and
// per channel Markstein's FMA correction: q0 = RN(a y), r = a - b q0 (exact with an FMA),
// q = RN(q0 + r y) (P. Markstein, "Computation of elementary functions on the IBM RISC
// System/6000 processor", IBM J. Res. Dev. 34(1), 1990).  Checked exhaustively against the
// IEEE division for every float a in [0, 8192) and every b = 1..31 (the whole range of
// w c + v and w + 1 here): q is the same bits for every a >= 2^-123; below that (where the
// residual r underflows) it can differ in the last place, and floor(q + 1/2) is the same
// for every a in the range.  The clamp to [0, 255] never binds, so it is not evaluated: the
// four tap weights are products of numbers in [0, 1] whose exact sum is 1, so the rounded
// sample v lies in [0, 255 (1 + 2^-21)], and with c <= 255 the quotient q stays below 255.5
// and at or above 0.
__device__ __forceinline__ unsigned blend_channel(unsigned c, float w, float v, float w1,
                                                  float rw1)
{
    const float a = fmaf(w, static_cast<float>(c), v);
    const float q0 = __fmul_rn(a, rw1);
    const float q = __fmaf_rn(__fmaf_rn(-q0, w1, a), rw1, q0);
    return static_cast<unsigned>(floorf(q + 0.5f));
}

// The update of one canvas pixel from its sample v, with rw1 = RN(1/(w + 1)) for the pixel's
// weight w (a kernel that updates many pixels may take it from a table of the 31 values).
template <int CH>
__device__ __forceinline__ uchar4 blend_update_r(uchar4 cv, const float (&v)[CH], float rw1)
{
    const float w = static_cast<float>(cv.w);
    const float w1 = w + 1.f;
    cv.x = blend_channel(cv.x, w, v[0], w1, rw1);
    if (CH == 3) {
        cv.y = blend_channel(cv.y, w, v[1 % CH], w1, rw1);
        cv.z = blend_channel(cv.z, w, v[2 % CH], w1, rw1);
    }
    cv.w = static_cast<unsigned char>(cv.w < 30 ? cv.w + 1 : 30);
    return cv;
}

template <int CH>
__device__ __forceinline__ uchar4 blend_update(uchar4 cv, const float (&v)[CH])
{
    return blend_update_r<CH>(cv, v, __frcp_rn(static_cast<float>(cv.w) + 1.f));
}

// One pixel: canvas pixel cp receives frame t sampled at p + d, or is left untouched.
template <int CH>
__device__ __forceinline__ void blend_pixel(const uint8_t *__restrict__ frame, int fw, int fh,
                                            int pitch, float px, float py, float dx, float dy,
                                            uchar4 *cp)
{
    const Tap t = tap_setup<CH>(fw, fh, pitch, px, py, dx, dy);
    if (!t.ok) return;
    float v[CH];
    tap_sample<CH>(frame, t, v);
    *cp = blend_update<CH>(*cp, v);
}

}  // namespace emdq
