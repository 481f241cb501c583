// Dense field on the CUDA cores in FP32: one thread per pixel, the matches streamed
// through shared memory (Eqs. 2-4 evaluated term by term, the paper's per-pixel GPU
// design).  Also the reference-warp reduction every field path starts with.
//
// Blend relative to a reference warp.  The blend is linear, so for any constant row
// Q_ref:  sum w_i Q_i / sum w_i = Q_ref + sum w_i (Q_i - Q_ref) / sum w_i.  Summing the
// small differences keeps FP32 rounding away from the scale and dual parts, which the
// pixel position (up to ~2000 px) multiplies.  Q_ref is the c-weighted mean row.
#include <cmath>

#include "common.cuh"
#include "field.cuh"

namespace emdq {

__global__ void __launch_bounds__(kRefThreads) field_ref_kernel(const float *__restrict__ q,
                                                                const float *__restrict__ c,
                                                                int n, float *__restrict__ ref)
{
    __shared__ float red[6 * 32];
    float r[6];
    reference_row(q, c, n, red, r);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) ref[k] = r[k];
}

// One thread per pixel of a 32 x 8 tile; matches in chunks of kDirectChunk through smem.
__global__ void __launch_bounds__(kDirectThreads) field_direct_kernel(
    const float *__restrict__ q, const float *__restrict__ c, const float2 *__restrict__ src,
    int n, int gx0, int gy0, int gw, int gh, float alpha, const float *__restrict__ ref,
    float2 *__restrict__ disp)
{
    __shared__ float sx[kDirectChunk], sy[kDirectChunk], sc[kDirectChunk];
    __shared__ float sa[kDirectChunk], sb[kDirectChunk], su[kDirectChunk], sv[kDirectChunk],
        ss[kDirectChunk];
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lx, y = blockIdx.y * 8 + ly;
    const float px = static_cast<float>(gx0 + x), py = static_cast<float>(gy0 + y);
    const float ra = ref[0], rb = ref[1], ru = ref[2], rv = ref[3], rs = ref[4];
    float w0 = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
    for (int base = 0; base < n; base += kDirectChunk) {
        const int m = min(kDirectChunk, n - base);
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += kDirectThreads) {
            const int i = base + k;
            const float2 xi = src[i];
            const float4 r0 = *reinterpret_cast<const float4 *>(q + 8 * (size_t)i);
            sx[k] = xi.x;
            sy[k] = xi.y;
            sc[k] = c[i];
            sa[k] = r0.x - ra;
            sb[k] = r0.y - rb;
            su[k] = r0.z - ru;
            sv[k] = r0.w - rv;
            ss[k] = q[8 * (size_t)i + 4] - rs;
        }
        __syncthreads();
        for (int k = 0; k < m; ++k) {
            const float dx = sx[k] - px, dy = sy[k] - py;
            const float w = sc[k] * expf(-alpha * (dx * dx + dy * dy));
            w0 += w;
            a0 += w * sa[k];
            a1 += w * sb[k];
            a2 += w * su[k];
            a3 += w * sv[k];
            a4 += w * ss[k];
        }
    }
    if (x >= gw || y >= gh) return;
    float2 d = make_float2(NAN, NAN);
    if (w0 > 0.f) {
        const float inv = 1.f / w0;
        const float2 xp = apply_blend(ra + a0 * inv, rb + a1 * inv, ru + a2 * inv, rv + a3 * inv,
                                      rs + a4 * inv, px, py);
        d = make_float2(xp.x - px, xp.y - py);
    }
    disp[(size_t)y * gw + x] = d;
}

}  // namespace emdq
