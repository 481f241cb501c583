// Field kernels shared between the translation units of libemdq.
#pragma once

#include "common.cuh"

namespace emdq {

constexpr int kRefThreads = 256;
constexpr int kDirectThreads = 256;   // 32 x 8 pixel tile
constexpr int kDirectChunk = 256;

// The blend reference row: the c-weighted mean warp row (r_w, r_z, d_x, d_y, s) of the
// first 256-row chunk that carries weight (any constant row is exact; the mean keeps the
// blended differences small).  Computed by a whole block (blockDim.x a multiple of 32,
// at most 1024) in a fixed order, so every block that calls it gets the same bits.
// red: shared scratch of 6 * 32 floats.  Returns the row in ref[0..4] of every thread;
// ref[5] is 1 if some match has weight, else 0 (and the row is the identity).
__device__ __forceinline__ void reference_row(const float *__restrict__ q, const float *__restrict__ c, int n,
                              float *red, float ref[6])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < n; base += 256) {
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int i = base + threadIdx.x; i < min(n, base + 256); i += blockDim.x) {
            const float ci = c[i];
            if (!(ci > 0.f)) continue;
            const float4 r0 = *reinterpret_cast<const float4 *>(q + 8 * (size_t)i);
            acc[0] += ci * r0.x;
            acc[1] += ci * r0.y;
            acc[2] += ci * r0.z;
            acc[3] += ci * r0.w;
            acc[4] += ci * q[8 * (size_t)i + 4];
            acc[5] += ci;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k)
            for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
        __syncthreads();
        if (lane == 0)
            for (int k = 0; k < 6; ++k) red[6 * w + k] = acc[k];
        __syncthreads();
        float t[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int ww = 0; ww < nw; ++ww)
            for (int k = 0; k < 6; ++k) t[k] += red[6 * ww + k];
        if (t[5] > 0.f) {
            for (int k = 0; k < 5; ++k) ref[k] = t[k] / t[5];
            ref[5] = 1.f;
            return;
        }
    }
    ref[0] = 1.f; ref[1] = 0.f; ref[2] = 0.f; ref[3] = 0.f; ref[4] = 1.f; ref[5] = 0.f;
}

__global__ void field_ref_kernel(const float *__restrict__ q, const float *__restrict__ c,
                                 int n, float *__restrict__ ref);

__global__ void field_direct_kernel(const float *__restrict__ q, const float *__restrict__ c,
                                    const float2 *__restrict__ src, int n, int gx0, int gy0,
                                    int gw, int gh, float alpha, const float *__restrict__ ref,
                                    float2 *__restrict__ disp);

}  // namespace emdq
