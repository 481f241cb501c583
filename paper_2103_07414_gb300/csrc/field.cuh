// Field kernels shared between the translation units of libemdq.
#pragma once

#include "common.cuh"

namespace emdq {

constexpr int kRefThreads = 256;
constexpr int kDirectThreads = 256;   // 32 x 8 pixel tile
constexpr int kDirectChunk = 256;

// The blend reference row: the c-weighted mean warp row (r_w, r_z, d_x, d_y, s) of the
// first 256-row chunk that carries weight (any constant row is exact; the mean keeps the
// blended differences small).  Summed by warp 0 in a fixed order (lane l adds rows l,
// l + 32, ... of the chunk, then a butterfly), so every block gets the same bits whatever
// its size (blockDim.x a multiple of 32).  red: shared scratch of at least 6 floats.
// Returns the row in ref[0..4] of every thread; ref[5] is 1 if some match has weight,
// else 0 (and the row is the identity).
__device__ __forceinline__ void reference_row(const float *__restrict__ q, const float *__restrict__ c, int n,
                              float *red, float ref[6])
{
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        float out[6] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f};
        for (int base = 0; base < n; base += 256) {
            // all loads of the chunk first (independent), then the sums in a fixed order
            float cw[8], r[8][5];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = base + lane + 32 * k;
                cw[k] = 0.f;
                r[k][0] = r[k][1] = r[k][2] = r[k][3] = r[k][4] = 0.f;
                if (i < n) {
                    cw[k] = c[i];
                    const float4 r0 = *reinterpret_cast<const float4 *>(q + 8 * (size_t)i);
                    r[k][0] = r0.x;
                    r[k][1] = r0.y;
                    r[k][2] = r0.z;
                    r[k][3] = r0.w;
                    r[k][4] = q[8 * (size_t)i + 4];
                }
            }
            float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (!(cw[k] > 0.f)) continue;         // weightless rows do not count
#pragma unroll
                for (int j = 0; j < 5; ++j) acc[j] += cw[k] * r[k][j];
                acc[5] += cw[k];
            }
#pragma unroll
            for (int k = 0; k < 6; ++k)
                for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
            if (acc[5] > 0.f) {          // the same decision in every lane
                for (int k = 0; k < 5; ++k) out[k] = acc[k] / acc[5];
                out[5] = 1.f;
                break;
            }
        }
        if (lane == 0)
            for (int k = 0; k < 6; ++k) red[k] = out[k];
    }
    __syncthreads();
    for (int k = 0; k < 6; ++k) ref[k] = red[k];
    __syncthreads();
}

__global__ void field_ref_kernel(const float *__restrict__ q, const float *__restrict__ c,
                                 int n, float *__restrict__ ref);

__global__ void field_direct_kernel(const float *__restrict__ q, const float *__restrict__ c,
                                    const float2 *__restrict__ src, int n, int gx0, int gy0,
                                    int gw, int gh, float alpha, const float *__restrict__ ref,
                                    float2 *__restrict__ disp);

}  // namespace emdq
