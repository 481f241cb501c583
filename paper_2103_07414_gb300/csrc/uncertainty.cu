// EMDQ uncertainty (Sec. III-C, Eq. 8): at every pixel p of the window, the minimum over the
// feature inliers j (the matches the fit keeps, c_j > 0) of exp(beta |p - x_j|^2), which is
// exp(beta d(p)^2) with d(p) the distance to the nearest inlier (exp increases for beta > 0).
// A block takes a 32 x 8 pixel tile.  It first finds the distance D0 from the tile centre o
// to its nearest inlier; the nearest inlier x* of any pixel p of the tile then lies within
// D0 + 2 r of o (r the tile's half-diagonal: |o - x*| <= |o - p| + |p - x*| <= r + |p - x0|
// <= 2 r + D0), so the inliers within that radius (plus half a pixel for rounding) are staged
// in shared memory as candidates and every pixel takes the minimum over them.
#include <cmath>

#include "common.cuh"

namespace emdq {

constexpr int kUncTX = 32, kUncTY = 8, kUncThreads = kUncTX * kUncTY;
constexpr int kUncCand = 2048;   // candidates staged per tile; beyond that, every inlier

__global__ void __launch_bounds__(kUncThreads) uncertainty_kernel(
    const float *__restrict__ c, const float2 *__restrict__ src, int n, int gx0, int gy0, int gw,
    int gh, float beta, float *__restrict__ out)
{
    __shared__ float2 cand[kUncCand];
    __shared__ int ncand;
    __shared__ float s_r2;
    const int tx0 = blockIdx.x * kUncTX, ty0 = blockIdx.y * kUncTY;
    const float ox = static_cast<float>(gx0 + tx0) + 0.5f * (kUncTX - 1);
    const float oy = static_cast<float>(gy0 + ty0) + 0.5f * (kUncTY - 1);
    const float r = 0.5f * sqrtf(static_cast<float>((kUncTX - 1) * (kUncTX - 1) +
                                                    (kUncTY - 1) * (kUncTY - 1)));
    __shared__ float wbest[kUncThreads / 32];
    {
        float best = INFINITY;
        for (int j = threadIdx.x; j < n; j += kUncThreads) {
            if (!(c[j] > 0.f)) continue;
            const float2 x = src[j];
            const float dx = x.x - ox, dy = x.y - oy;
            best = fminf(best, dx * dx + dy * dy);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
        if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kUncThreads / 32; ++w) best = fminf(best, wbest[w]);
            const float R = sqrtf(best) + 2.f * r + 0.5f;
            s_r2 = R * R;                       // +inf without inliers
            ncand = 0;
        }
    }
    __syncthreads();
    const float r2 = s_r2;
    for (int j = threadIdx.x; j < n; j += kUncThreads) {
        if (!(c[j] > 0.f)) continue;
        const float2 x = src[j];
        const float dx = x.x - ox, dy = x.y - oy;
        if (dx * dx + dy * dy <= r2) {
            const int k = atomicAdd(&ncand, 1);
            if (k < kUncCand) cand[k] = x;
        }
    }
    __syncthreads();
    const int m = ncand;
    const int x = tx0 + static_cast<int>(threadIdx.x) % kUncTX;
    const int y = ty0 + static_cast<int>(threadIdx.x) / kUncTX;
    const float px = static_cast<float>(gx0 + x), py = static_cast<float>(gy0 + y);
    float d2 = INFINITY;
    if (m <= kUncCand) {
        for (int k = 0; k < m; ++k) {
            const float2 q = cand[k];
            const float dx = q.x - px, dy = q.y - py;
            d2 = fminf(d2, dx * dx + dy * dy);
        }
    } else {
        for (int j = 0; j < n; ++j) {
            if (!(c[j] > 0.f)) continue;
            const float2 q = src[j];
            const float dx = q.x - px, dy = q.y - py;
            d2 = fminf(d2, dx * dx + dy * dy);
        }
    }
    if (x < gw && y < gh) out[(size_t)y * gw + x] = expf(beta * d2);
}

}  // namespace emdq

using namespace emdq;
using namespace emdq_host;

extern "C" emdq_status emdq_uncertainty(const float *c, const float *src, int n, int grid_x0,
                                        int grid_y0, int grid_w, int grid_h, float beta,
                                        float *out, void *stream)
{
    if (n < 0 || grid_w < 0 || grid_h < 0 || !(beta > 0.f) || !std::isfinite(beta))
        return EMDQ_EINVAL;
    if (grid_w == 0 || grid_h == 0) return EMDQ_OK;
    if (!out || (n > 0 && (!c || !src || !aligned(src, 8)))) return EMDQ_EINVAL;
    if ((grid_h + kUncTY - 1) / kUncTY > 65535) return EMDQ_ENOTSUP;
    const dim3 grid((grid_w + kUncTX - 1) / kUncTX, (grid_h + kUncTY - 1) / kUncTY);
    uncertainty_kernel<<<grid, kUncThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        c, reinterpret_cast<const float2 *>(src), n, grid_x0, grid_y0, grid_w, grid_h, beta, out);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}
