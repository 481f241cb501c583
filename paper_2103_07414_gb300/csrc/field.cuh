// Field kernels shared between the translation units of libemdq.
#pragma once

#include "common.cuh"

namespace emdq {

constexpr int kRefThreads = 256;
constexpr int kDirectThreads = 256;   // 32 x 8 pixel tile
constexpr int kDirectChunk = 256;

// ref[0..4]: c-weighted mean warp row (r_w, r_z, d_x, d_y, s); ref[5]: 1 if any weight.
__global__ void field_ref_kernel(const float *__restrict__ q, const float *__restrict__ c,
                                 int n, float *__restrict__ ref);

__global__ void field_direct_kernel(const float *__restrict__ q, const float *__restrict__ c,
                                    const float2 *__restrict__ src, int n, int gx0, int gy0,
                                    int gw, int gh, float alpha, const float *__restrict__ ref,
                                    float2 *__restrict__ disp);

}  // namespace emdq
