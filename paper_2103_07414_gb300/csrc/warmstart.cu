// Learned EM warm start: per-match nearest-neighbour residual features, a 16-64-64-1
// network with BF16 operands and FP32 accumulation that predicts each match's initial
// inlier weight p0, and the kernels that train it (forward, backward, Adam).
//
// Features of match j: its 8 nearest matches k != j by |x_k - x_j| (float32 squared
// distances, ties to the lower index); f1_k = log(1 + |(y_k - x_k) - (y_j - x_j)|) (the
// residual of k under the translation j implies: needs no fit, so it stays informative
// with many outliers) and f2_k = log(1 + |x_k - x_j|) (the distance, the scale for
// judging those residuals), in pixels, each group sorted ascending.  Parameters (5313 floats): W1[64][16], b1[64], W2[64][64],
// b2[64], W3[64], b3.  The forward rounds parameters, inputs and hidden activations to
// BF16 and accumulates in FP32; training keeps FP32 master weights.
#include <cuda_bf16.h>

#include "common.cuh"

namespace emdq {

constexpr int kKnn = 8;
constexpr int kNin = 16, kNh = 64;
constexpr int kOffW1 = 0, kOffB1 = kNh * kNin, kOffW2 = kOffB1 + kNh, kOffB2 = kOffW2 + kNh * kNh,
              kOffW3 = kOffB2 + kNh, kOffB3 = kOffW3 + kNh, kNParams = kOffB3 + 1;
static_assert(kNParams == 5313, "parameter layout");

constexpr int kMlpThreads = 128;      // also the samples of one training tile

__device__ __forceinline__ float bf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// ------------------------------------------------------------------ features ----------
// One warp per match.  Each lane keeps the 8 nearest of the candidates it is offered,
// sorted by (distance, index); 8 rounds of a warp-wide lexicographic arg-min then pop the
// overall 8 nearest in order -- the same set and order as a full sort.  All lanes end with
// the 16 features.
struct Near8 {
    float d[kKnn];
    int i[kKnn];
};

__device__ __forceinline__ void near8_reset(Near8 &L)
{
#pragma unroll
    for (int k = 0; k < kKnn; ++k) {
        L.d[k] = INFINITY;
        L.i[k] = 0x7fffffff;
    }
}

__device__ __forceinline__ bool near8_before(float d, int i, float e, int k)
{
    return d < e || (d == e && i < k);
}

// float32, one rounding per operation (the same decision as the oracle's)
__device__ __forceinline__ float near_d2(float2 xi, float2 xj)
{
    const float dx = __fsub_rn(xi.x, xj.x), dy = __fsub_rn(xi.y, xj.y);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

__device__ __forceinline__ void near8_offer(Near8 &L, float d, int i)
{
    if (!near8_before(d, i, L.d[kKnn - 1], L.i[kKnn - 1])) return;
    float cd = d;
    int ci = i;
#pragma unroll
    for (int s = 0; s < kKnn; ++s) {
        const bool lt = near8_before(cd, ci, L.d[s], L.i[s]);
        const float td = L.d[s];
        const int ti = L.i[s];
        if (lt) {
            L.d[s] = cd;
            L.i[s] = ci;
            cd = td;
            ci = ti;
        }
    }
}

// The warp's 8 nearest over all lanes' lists, ascending (consumes the lists).
__device__ __forceinline__ void near8_merge(Near8 &L, float (&nd)[kKnn], int (&ni)[kKnn])
{
    // round r: the least (d, i) of the lanes' heads.  Squared distances are +0 or positive
    // (NaN is never kept, empty slots are +inf), so their bits order as unsigned integers:
    // the warp minimum of the bits, then the least index among the lanes that hold it
#pragma unroll
    for (int r = 0; r < kKnn; ++r) {
        const unsigned hb = __float_as_uint(L.d[0]);
        const unsigned mb = __reduce_min_sync(0xffffffffu, hb);
        const int ci = static_cast<int>(__reduce_min_sync(
            0xffffffffu, hb == mb ? static_cast<unsigned>(L.i[0]) : 0xffffffffu));
        const float cd = __uint_as_float(mb);
        nd[r] = cd;
        ni[r] = ci;
        if (L.i[0] == ci) {          // this lane held the winner: pop its head
#pragma unroll
            for (int s = 0; s + 1 < kKnn; ++s) {
                L.d[s] = L.d[s + 1];
                L.i[s] = L.i[s + 1];
            }
            L.d[kKnn - 1] = INFINITY;
            L.i[kKnn - 1] = 0x7fffffff;
        }
    }
}

// The 16 features of match j from its 8 nearest (nd ascending, indices ni).
__device__ __forceinline__ void near8_features(const float2 *__restrict__ src,
                                               const float2 *__restrict__ dst, int j,
                                               int n, const float (&nd)[kKnn],
                                               const int (&ni)[kKnn], int lane,
                                               float (&f)[2 * kKnn])
{
    // lane k < 8: the residual of neighbour k under the translation match j implies.  A
    // missing neighbour (non-finite coordinates compare false, so fewer than 8 may be
    // found) gives a NaN feature, which the fit then reports as a non-finite p0.
    const float2 xj = src[j], yj = dst[j];
    const float djx = yj.x - xj.x, djy = yj.y - xj.y;
    float mine = 0.f;
    if (lane < kKnn) {
        int idx = ni[0];
#pragma unroll
        for (int k = 1; k < kKnn; ++k)
            if (lane == k) idx = ni[k];
        if (idx >= 0 && idx < n) {
            const float2 xk = src[idx], yk = dst[idx];
            mine = log1pf(hypotf((yk.x - xk.x) - djx, (yk.y - xk.y) - djy));
        } else {
            mine = __int_as_float(0x7fffffff);
        }
    }
    float f1[kKnn];
#pragma unroll
    for (int k = 0; k < kKnn; ++k) f1[k] = __shfl_sync(0xffffffffu, mine, k);
    // sort ascending (odd-even transposition, fixed network; every lane the same)
#pragma unroll
    for (int r = 0; r < kKnn; ++r)
#pragma unroll
        for (int k = r & 1; k + 1 < kKnn; k += 2) {
            const float lo = fminf(f1[k], f1[k + 1]), hi = fmaxf(f1[k], f1[k + 1]);
            f1[k] = lo;
            f1[k + 1] = hi;
        }
    // the distances (already ascending): lane k < 8 takes the k-th, all lanes get all 8
    float dk = nd[0];
#pragma unroll
    for (int k = 1; k < kKnn; ++k)
        if (lane == k) dk = nd[k];
    const float lk = log1pf(sqrtf(dk));
#pragma unroll
    for (int k = 0; k < kKnn; ++k) {
        f[k] = f1[k];
        f[kKnn + k] = __shfl_sync(0xffffffffu, lk, k);
    }
}

// Brute force: every match is a candidate (lane l takes i = l + 32 t).
__device__ __forceinline__ void knn_features_warp(const float2 *__restrict__ src,
                                                  const float2 *__restrict__ dst, int n, int j,
                                                  int lane, float (&f)[2 * kKnn])
{
    const float2 xj = src[j];
    Near8 L;
    near8_reset(L);
    for (int i = lane; i < n; i += 32)
        if (i != j) near8_offer(L, near_d2(src[i], xj), i);
    float nd[kKnn];
    int ni[kKnn];
    near8_merge(L, nd, ni);
    near8_features(src, dst, j, n, nd, ni, lane, f);
}

__global__ void __launch_bounds__(256) warm_features_kernel(const float2 *__restrict__ src,
                                                           const float2 *__restrict__ dst, int n,
                                                           float *__restrict__ feat)
{
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += nw) {
        float f[2 * kKnn];
        knn_features_warp(src, dst, n, j, lane, f);
        if (lane < 2 * kKnn) {
            float v = f[0];
#pragma unroll
            for (int k = 1; k < 2 * kKnn; ++k)
                if (lane == k) v = f[k];
            feat[16 * (size_t)j + lane] = v;
        }
    }
}

// ------------------------------------------------------------------ network ------------
// Parameters rounded to BF16, staged in shared memory as floats: W1 and W2 by output row
// ([out][in]), each row padded to a multiple of 4 floats plus 4, so that the lanes' 16-byte
// reads of four inputs of their own rows fall in distinct banks; then per warp 64 floats for the
// hidden layer (every lane reads its values by broadcast).
constexpr int kSwLd1 = kNin + 4, kSwLd2 = kNh + 4;
constexpr int kSwW1 = 0, kSwB1 = kSwW1 + kNh * kSwLd1, kSwW2 = kSwB1 + kNh,
              kSwB2 = kSwW2 + kNh * kSwLd2, kSwW3 = kSwB2 + kNh, kSwB3 = kSwW3 + kNh,
              kSwH = (kSwB3 + 1 + 3) / 4 * 4;
static_assert(kSwW1 % 4 == 0 && kSwW2 % 4 == 0 && kSwLd1 % 4 == 0 && kSwLd2 % 4 == 0, "16-byte rows");

// Parameters rounded to BF16 in their stored layout (for the training kernel).
__device__ __forceinline__ void stage_params(const float *__restrict__ w, float *sw)
{
    for (int k = threadIdx.x; k < kNParams; k += blockDim.x) sw[k] = bf(w[k]);
    __syncthreads();
}

__device__ __forceinline__ void stage_params_t(const float *__restrict__ w, float *sw)
{
    for (int k = threadIdx.x; k < kNParams; k += blockDim.x) {
        const float v = bf(w[k]);
        int d;
        if (k < kOffB1) d = kSwW1 + (k / kNin) * kSwLd1 + k % kNin;                 // W1[o][m]
        else if (k < kOffW2) d = kSwB1 + (k - kOffB1);
        else if (k < kOffB2) d = kSwW2 + ((k - kOffW2) / kNh) * kSwLd2 + (k - kOffW2) % kNh;
        else if (k < kOffW3) d = kSwB2 + (k - kOffB2);
        else if (k < kOffB3) d = kSwW3 + (k - kOffW3);
        else d = kSwB3;
        sw[d] = v;
    }
    __syncthreads();
}

// One sample per warp: lane l computes hidden units l and l + 32 of both layers; inputs
// rounded to BF16, FP32 accumulation in input order; returns the logit z in every lane.  hs:
// this warp's 64 floats of shared scratch (the first hidden layer, read by broadcast).
__device__ __forceinline__ float mlp_forward_warp(const float *sw, const float (&f)[2 * kKnn],
                                                  int lane, float *hs)
{
    float x[kNin];
#pragma unroll
    for (int m = 0; m < kNin; ++m) x[m] = bf(f[m]);
    float a0 = sw[kSwB1 + lane], a1 = sw[kSwB1 + lane + 32];
    const float *r0 = sw + kSwW1 + lane * kSwLd1, *r1 = sw + kSwW1 + (lane + 32) * kSwLd1;
#pragma unroll
    for (int m = 0; m < kNin; m += 4) {
        const float4 u = *reinterpret_cast<const float4 *>(r0 + m);
        const float4 v = *reinterpret_cast<const float4 *>(r1 + m);
        a0 = fmaf(u.x, x[m], a0);
        a0 = fmaf(u.y, x[m + 1], a0);
        a0 = fmaf(u.z, x[m + 2], a0);
        a0 = fmaf(u.w, x[m + 3], a0);
        a1 = fmaf(v.x, x[m], a1);
        a1 = fmaf(v.y, x[m + 1], a1);
        a1 = fmaf(v.z, x[m + 2], a1);
        a1 = fmaf(v.w, x[m + 3], a1);
    }
    hs[lane] = bf(fmaxf(a0, 0.f));
    hs[lane + 32] = bf(fmaxf(a1, 0.f));
    __syncwarp();
    float c0 = sw[kSwB2 + lane], c1 = sw[kSwB2 + lane + 32];
    const float *q0 = sw + kSwW2 + lane * kSwLd2, *q1 = sw + kSwW2 + (lane + 32) * kSwLd2;
#pragma unroll
    for (int k = 0; k < kNh; k += 4) {
        const float4 h = *reinterpret_cast<const float4 *>(hs + k);
        const float4 u = *reinterpret_cast<const float4 *>(q0 + k);
        const float4 v = *reinterpret_cast<const float4 *>(q1 + k);
        c0 = fmaf(u.x, h.x, c0);
        c0 = fmaf(u.y, h.y, c0);
        c0 = fmaf(u.z, h.z, c0);
        c0 = fmaf(u.w, h.w, c0);
        c1 = fmaf(v.x, h.x, c1);
        c1 = fmaf(v.y, h.y, c1);
        c1 = fmaf(v.z, h.z, c1);
        c1 = fmaf(v.w, h.w, c1);
    }
    __syncwarp();                           // the scratch is free for the next sample
    float z = sw[kSwW3 + lane] * bf(fmaxf(c0, 0.f)) + sw[kSwW3 + lane + 32] * bf(fmaxf(c1, 0.f));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    return z + sw[kSwB3];
}

constexpr int kNetThreads = 256;
constexpr int kSwTotal = kSwH + 64 * (kNetThreads / 32);   // staged network + hidden scratch

__global__ void __launch_bounds__(kNetThreads) warm_infer_kernel(const float *__restrict__ feat,
                                                                 int n, const float *__restrict__ w,
                                                                 float *__restrict__ p0)
{
    __shared__ __align__(16) float sw[kSwTotal];
    stage_params_t(w, sw);
    const int lane = threadIdx.x & 31;
    float *hs = sw + kSwH + 64 * (threadIdx.x >> 5);
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += nw) {
        float f[2 * kKnn];
#pragma unroll
        for (int m = 0; m < 2 * kKnn; ++m) f[m] = feat[16 * (size_t)j + m];
        const float z = mlp_forward_warp(sw, f, lane, hs);
        if (lane == 0) p0[j] = 1.f / (1.f + expf(-z));
    }
}

// Features + network for many problems in one launch, one warp per match.
constexpr int kWarmBatchMax = 64;
struct WarmBatch {
    const float2 *src[kWarmBatchMax];
    const float2 *dst[kWarmBatchMax];
    float *p0[kWarmBatchMax];
    int n[kWarmBatchMax];
    int first[kWarmBatchMax + 1];       // prefix sums of the problems' match counts
    int count;
};

__global__ void __launch_bounds__(kNetThreads) warm_start_batch_kernel(
    const __grid_constant__ WarmBatch B, const float *__restrict__ w)
{
    __shared__ __align__(16) float sw[kSwTotal];
    stage_params_t(w, sw);
    const int lane = threadIdx.x & 31;
    float *hs = sw + kSwH + 64 * (threadIdx.x >> 5);
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int total = B.first[B.count];
    int b = 0;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < total; g += nw) {
        while (g >= B.first[b + 1]) ++b;       // g only grows
        const int j = g - B.first[b];
        float f[2 * kKnn];
        knn_features_warp(B.src[b], B.dst[b], B.n[b], j, lane, f);
        const float z = mlp_forward_warp(sw, f, lane, hs);
        if (lane == 0) B.p0[b][j] = 1.f / (1.f + expf(-z));
    }
}

// The same p0 by a kNN search that visits few candidates.  A block takes up to
// kGridQueries matches of one problem and first stages all of that problem's matches in
// shared memory, bucketed by a uniform grid of square cells (about kGridPerCell matches per
// cell).  A warp offers its match the matches of the 3 x 3 cells around its own.  When the
// 8th nearest found is closer than the edge of that block of cells (with a margin that
// covers the rounding of the cell assignment), no match outside it can be among the 8
// nearest and the result is final; otherwise a larger block is searched, bounded by the
// 8th nearest found, until that holds or the block is the whole grid.  The result is the 8
// nearest by (distance, index): the set and order of the brute-force search, so the
// features and p0 are the same bits.
constexpr int kGridMaxN = 8192;        // matches staged per block (indices fit 16 bits)
constexpr int kGridCells = 2048;
constexpr float kGridPerCell = 8.f;
constexpr int kGridQueries = 128;      // matches per block, 16 per warp

struct WarmGridBatch {
    const float2 *src[kWarmBatchMax];
    const float2 *dst[kWarmBatchMax];
    float *p0[kWarmBatchMax];
    int n[kWarmBatchMax];
    int block0[kWarmBatchMax + 1];     // prefix sums of the problems' block counts
    int count;
    int nmax;                          // largest n (sizes the shared-memory arrays)
    int queries;                       // matches per block (kGridQueries, fewer for small launches)
};

struct GridLayout {
    size_t pts, idx, start, cur, misc, total;
};

__host__ __device__ inline size_t al16(size_t v) { return (v + 15) / 16 * 16; }

__host__ __device__ inline GridLayout grid_layout(int nmax)
{
    GridLayout L;
    L.pts = al16(sizeof(float) * kSwTotal);
    L.idx = L.pts + al16(sizeof(float2) * (size_t)nmax);
    L.start = L.idx + al16(sizeof(unsigned short) * (size_t)nmax);
    L.cur = L.start + al16(sizeof(int) * (kGridCells + 1));
    L.misc = L.cur + al16(sizeof(int) * kGridCells);
    L.total = L.misc + al16(sizeof(float) * 48);
    return L;
}

struct GridGeom {
    float x0, y0, c, inv_c;
    int gx, gy;
};

__device__ __forceinline__ int grid_cell(const GridGeom &G, float2 x, int &cx, int &cy)
{
    cx = min(max(static_cast<int>((x.x - G.x0) * G.inv_c), 0), G.gx - 1);
    cy = min(max(static_cast<int>((x.y - G.y0) * G.inv_c), 0), G.gy - 1);
    return cy * G.gx + cx;
}

__global__ void __launch_bounds__(kNetThreads) warm_start_grid_kernel(
    const __grid_constant__ WarmGridBatch B, const float *__restrict__ w)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const GridLayout SL = grid_layout(B.nmax);
    float *sw = reinterpret_cast<float *>(smem);
    float *hs = sw + kSwH + 64 * (threadIdx.x >> 5);
    float2 *pts = reinterpret_cast<float2 *>(smem + SL.pts);
    unsigned short *idx = reinterpret_cast<unsigned short *>(smem + SL.idx);
    int *start = reinterpret_cast<int *>(smem + SL.start);
    int *cur = reinterpret_cast<int *>(smem + SL.cur);
    float *misc = reinterpret_cast<float *>(smem + SL.misc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = kNetThreads / 32;

    int b = 0;
    while (b + 1 < B.count && static_cast<int>(blockIdx.x) >= B.block0[b + 1]) ++b;
    const int n = B.n[b];
    const float2 *__restrict__ src = B.src[b];
    const int q0 = (blockIdx.x - B.block0[b]) * B.queries;

    for (int k = threadIdx.x; k < kGridCells; k += kNetThreads) cur[k] = 0;
    // extent of the matches (NaNs are ignored by fminf / fmaxf)
    float mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
    for (int i = threadIdx.x; i < n; i += kNetThreads) {
        const float2 x = src[i];
        mnx = fminf(mnx, x.x);
        mny = fminf(mny, x.y);
        mxx = fmaxf(mxx, x.x);
        mxy = fmaxf(mxy, x.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    }
    if (lane == 0) {
        misc[4 * warp + 0] = mnx;
        misc[4 * warp + 1] = mny;
        misc[4 * warp + 2] = mxx;
        misc[4 * warp + 3] = mxy;
    }
    stage_params_t(w, sw);                 // ends with __syncthreads
    if (threadIdx.x == 0) {
        for (int k = 1; k < kWarps; ++k) {
            mnx = fminf(mnx, misc[4 * k + 0]);
            mny = fminf(mny, misc[4 * k + 1]);
            mxx = fmaxf(mxx, misc[4 * k + 2]);
            mxy = fmaxf(mxy, misc[4 * k + 3]);
        }
        const float wx = mxx - mnx, wy = mxy - mny;
        GridGeom G{mnx, mny, 1.f, 1.f, 1, 1};
        if (isfinite(wx) && isfinite(wy)) {
            // square cells of about kGridPerCell matches (a line of matches: by its length)
            float c = sqrtf(wx * wy * kGridPerCell / n);
            c = fmaxf(c, fmaxf(wx, wy) * kGridPerCell / n);
            c = fmaxf(c, 1e-3f);
            for (;;) {
                G.gx = static_cast<int>(wx / c) + 1;
                G.gy = static_cast<int>(wy / c) + 1;
                if (G.gx * G.gy <= kGridCells) break;
                c *= 1.25f;
            }
            G.c = c;
            G.inv_c = 1.f / c;
        } else {
            G.x0 = G.y0 = 0.f;             // one cell: every search is the whole problem
        }
        *reinterpret_cast<GridGeom *>(misc + 32) = G;
    }
    __syncthreads();
    const GridGeom G = *reinterpret_cast<const GridGeom *>(misc + 32);
    int cx, cy;
    for (int i = threadIdx.x; i < n; i += kNetThreads) atomicAdd(&cur[grid_cell(G, src[i], cx, cy)], 1);
    __syncthreads();
    // exclusive scan of the cell counts into start[0 .. kGridCells]
    {
        constexpr int per = kGridCells / kNetThreads;
        int v[per], sum = 0;
#pragma unroll
        for (int u = 0; u < per; ++u) {
            v[u] = cur[threadIdx.x * per + u];
            sum += v[u];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int *wsum = reinterpret_cast<int *>(misc);          // the extents are no longer needed
        __syncthreads();
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int off = incl - sum;
        for (int k = 0; k < warp; ++k) off += wsum[k];
#pragma unroll
        for (int u = 0; u < per; ++u) {
            start[threadIdx.x * per + u] = off;
            cur[threadIdx.x * per + u] = off;
            off += v[u];
        }
        if (threadIdx.x == kNetThreads - 1) start[kGridCells] = off;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kNetThreads) {
        const float2 x = src[i];
        const int pos = atomicAdd(&cur[grid_cell(G, x, cx, cy)], 1);
        pts[pos] = x;
        idx[pos] = static_cast<unsigned short>(i);
    }
    __syncthreads();

    for (int k = warp; k < B.queries; k += kWarps) {
        const int j = q0 + k;
        if (j >= n) break;
        const float2 xj = src[j];
        grid_cell(G, xj, cx, cy);
        // blocks of (2R + 1)^2 cells around x_j, R = 1, 2, 4, ..., each searched afresh with
        // the previous block's 8th nearest as the bound, until the 8th nearest is closer
        // than every cell outside the block
        float nd[kKnn], td = INFINITY;
        int ni[kKnn], ti = 0x7fffffff;
        for (int R = 1;; R = R < 2 ? R + 1 : 2 * R) {
            const int xl = max(cx - R, 0), xh = min(cx + R, G.gx - 1);
            const int yl = max(cy - R, 0), yh = min(cy + R, G.gy - 1);
            Near8 L;
            near8_reset(L);
            for (int row = yl; row <= yh; ++row) {
                const int e = start[row * G.gx + xh + 1];
                for (int t = start[row * G.gx + xl] + lane; t < e; t += 32) {
                    const int i = idx[t];
                    if (i == j) continue;
                    const float d = near_d2(pts[t], xj);
                    if (!near8_before(td, ti, d, i)) near8_offer(L, d, i);
                }
            }
            near8_merge(L, nd, ni);
            // distance from x_j to the nearest block edge that has cells beyond it
            float bnd = INFINITY;
            if (xl > 0) bnd = fminf(bnd, xj.x - (G.x0 + xl * G.c));
            if (xh < G.gx - 1) bnd = fminf(bnd, (G.x0 + (xh + 1) * G.c) - xj.x);
            if (yl > 0) bnd = fminf(bnd, xj.y - (G.y0 + yl * G.c));
            if (yh < G.gy - 1) bnd = fminf(bnd, (G.y0 + (yh + 1) * G.c) - xj.y);
            const float r = bnd * 0.999f - 0.01f;
            if (bnd == INFINITY || (r > 0.f && nd[kKnn - 1] < r * r)) break;
            td = nd[kKnn - 1];          // itself a candidate (so <= passes), or still INF
            ti = ni[kKnn - 1];
        }
        float f[2 * kKnn];
        near8_features(src, B.dst[b], j, n, nd, ni, lane, f);
        const float z = mlp_forward_warp(sw, f, lane, hs);
        if (lane == 0) B.p0[b][j] = 1.f / (1.f + expf(-z));
    }
}

// Gradient of the summed cross-entropy over one tile of kMlpThreads samples, written as
// the tile's partial (kNParams floats) plus its loss sum (one float).  Per-sample terms
// are kept in shared memory as [feature][sample] (row stride kLd, padded against bank
// conflicts); the weight gradients are then sums over the tile's samples.  The gradient
// is that of the BF16-rounded network, applied to the FP32 master weights.
constexpr int kLd = kMlpThreads + 1;

__global__ void __launch_bounds__(kMlpThreads) mlp_grad_kernel(
    const float *__restrict__ feat, const float *__restrict__ label, int batch,
    const float *__restrict__ w, float *__restrict__ partial)
{
    extern __shared__ float sm[];
    float *sw = sm;                       // kNParams
    float *sx = sw + kNParams;            // [kNin][kLd]  x (rounded)
    float *sh1 = sx + kNin * kLd;         // [kNh][kLd]   h1 (rounded)
    float *sh2 = sh1 + kNh * kLd;         // [kNh][kLd]   h2 (rounded)
    float *sd2 = sh2 + kNh * kLd;         // [kNh][kLd]   dL/da2
    float *sd1 = sd2 + kNh * kLd;         // [kNh][kLd]   dL/da1
    float *sdz = sd1 + kNh * kLd;         // [kMlpThreads] dL/dz
    float *sloss = sdz + kMlpThreads;     // [kMlpThreads]
    stage_params(w, sw);
    const int t = threadIdx.x;
    const int s = blockIdx.x * kMlpThreads + t;
    const bool live = s < batch;
    float x[kNin], h1[kNh];
#pragma unroll
    for (int m = 0; m < kNin; ++m) {
        x[m] = live ? bf(feat[16 * (size_t)s + m]) : 0.f;
        sx[m * kLd + t] = x[m];
    }
#pragma unroll
    for (int o = 0; o < kNh; ++o) {
        float acc = sw[kOffB1 + o];
#pragma unroll
        for (int m = 0; m < kNin; ++m) acc = fmaf(sw[kOffW1 + o * kNin + m], x[m], acc);
        h1[o] = bf(fmaxf(acc, 0.f));
        sh1[o * kLd + t] = h1[o];
    }
    float z = sw[kOffB3];
#pragma unroll 1
    for (int o = 0; o < kNh; ++o) {
        float acc = sw[kOffB2 + o];
#pragma unroll
        for (int k = 0; k < kNh; ++k) acc = fmaf(sw[kOffW2 + o * kNh + k], h1[k], acc);
        const float h2 = bf(fmaxf(acc, 0.f));
        sh2[o * kLd + t] = h2;
        sd2[o * kLd + t] = acc;              // pre-activation, turned into dL/da2 below
        z = fmaf(sw[kOffW3 + o], h2, z);
    }
    const float y = live ? label[s] : 0.f;
    const float p = 1.f / (1.f + expf(-z));
    const float dz = live ? p - y : 0.f;
    sloss[t] = live ? (fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))) - y * z) : 0.f;   // softplus(z) - y z
    sdz[t] = dz;
    for (int o = 0; o < kNh; ++o)
        sd2[o * kLd + t] = sd2[o * kLd + t] > 0.f ? dz * sw[kOffW3 + o] : 0.f;
    for (int k = 0; k < kNh; ++k) {
        float acc = 0.f;
        for (int o = 0; o < kNh; ++o) acc = fmaf(sw[kOffW2 + o * kNh + k], sd2[o * kLd + t], acc);
        sd1[k * kLd + t] = sh1[k * kLd + t] > 0.f ? acc : 0.f;   // h1 > 0 exactly when a1 > 0
    }
    __syncthreads();
    float *out = partial + (size_t)blockIdx.x * (kNParams + 1);
    for (int q = t; q < kNParams + 1; q += kMlpThreads) {
        float acc = 0.f;
        if (q < kOffB1) {                           // W1[o][m]
            const int o = q / kNin, m = q % kNin;
            for (int r = 0; r < kMlpThreads; ++r) acc = fmaf(sd1[o * kLd + r], sx[m * kLd + r], acc);
        } else if (q < kOffW2) {                    // b1
            const int o = q - kOffB1;
            for (int r = 0; r < kMlpThreads; ++r) acc += sd1[o * kLd + r];
        } else if (q < kOffB2) {                    // W2[o][k]
            const int o = (q - kOffW2) / kNh, k = (q - kOffW2) % kNh;
            for (int r = 0; r < kMlpThreads; ++r) acc = fmaf(sd2[o * kLd + r], sh1[k * kLd + r], acc);
        } else if (q < kOffW3) {                    // b2
            const int o = q - kOffB2;
            for (int r = 0; r < kMlpThreads; ++r) acc += sd2[o * kLd + r];
        } else if (q < kOffB3) {                    // W3
            const int o = q - kOffW3;
            for (int r = 0; r < kMlpThreads; ++r) acc = fmaf(sdz[r], sh2[o * kLd + r], acc);
        } else if (q == kOffB3) {                   // b3
            for (int r = 0; r < kMlpThreads; ++r) acc += sdz[r];
        } else {                                    // loss sum
            for (int r = 0; r < kMlpThreads; ++r) acc += sloss[r];
        }
        out[q] = acc;
    }
}

constexpr size_t kGradSmem =
    sizeof(float) * (kNParams + kNin * kLd + 4 * kNh * kLd + 2 * kMlpThreads);

// Mean gradient over the batch from the tile partials (fixed order), then optionally one
// Adam step of the FP32 master weights.  Also writes the mean loss and the gradient.
__global__ void mlp_adam_kernel(const float *__restrict__ partial, int tiles, int batch,
                                float *__restrict__ w, float *__restrict__ m,
                                float *__restrict__ v, float *__restrict__ g_out,
                                float *__restrict__ loss_out, int step, float lr, float b1,
                                float b2, float eps, int update)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > kNParams) return;
    float acc = 0.f;
    for (int c = 0; c < tiles; ++c) acc += partial[(size_t)c * (kNParams + 1) + q];
    const float g = acc / static_cast<float>(batch);
    if (q == kNParams) {
        if (loss_out) *loss_out = g;
        return;
    }
    if (g_out) g_out[q] = g;
    if (!update) return;
    const float mq = b1 * m[q] + (1.f - b1) * g;
    const float vq = b2 * v[q] + (1.f - b2) * g * g;
    m[q] = mq;
    v[q] = vq;
    const float mh = mq / (1.f - powf(b1, static_cast<float>(step)));
    const float vh = vq / (1.f - powf(b2, static_cast<float>(step)));
    w[q] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace emdq

using namespace emdq;
using namespace emdq_host;

extern "C" int emdq_mlp_param_count(void) { return kNParams; }

extern "C" emdq_status emdq_warm_features(const float *src, const float *dst, int n,
                                          float *feat_out, void *stream)
{
    if (!src || !dst || !feat_out || n < kKnn + 1) return EMDQ_EINVAL;
    if (!aligned(src, 8) || !aligned(dst, 8) || !aligned(feat_out, 16))
        return EMDQ_EINVAL;
    const int blocks = (n + 7) / 8 < 1024 ? (n + 7) / 8 : 1024;    // 8 warps per block
    warm_features_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float2 *>(src), reinterpret_cast<const float2 *>(dst), n, feat_out);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

extern "C" emdq_status emdq_warm_infer(const float *feat, int n, const float *params,
                                       float *p0_out, void *stream)
{
    if (!feat || !params || !p0_out || n < 1) return EMDQ_EINVAL;
    const DeviceInfo &D = device_info();
    const int want = (n + 7) / 8, cap = 2 * (D.sms > 0 ? D.sms : 152);
    warm_infer_kernel<<<want < cap ? want : cap, kNetThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        feat, n, params, p0_out);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

extern "C" emdq_status emdq_warm_start(const float *const *src, const float *const *dst,
                                       const int *n, float *const *p0_out, int count,
                                       const float *params, void *stream)
{
    if (!src || !dst || !n || !p0_out || !params || count < 1) return EMDQ_EINVAL;
    if (count > kWarmBatchMax) return EMDQ_ENOTSUP;
    WarmBatch B;
    B.count = count;
    int total = 0;
    for (int b = 0; b < count; ++b) {
        if (!src[b] || !dst[b] || !p0_out[b] || n[b] < kKnn + 1) return EMDQ_EINVAL;
        if (!aligned(src[b], 8) || !aligned(dst[b], 8)) return EMDQ_EINVAL;
        B.src[b] = reinterpret_cast<const float2 *>(src[b]);
        B.dst[b] = reinterpret_cast<const float2 *>(dst[b]);
        B.p0[b] = p0_out[b];
        B.n[b] = n[b];
        B.first[b] = total;
        total += n[b];
    }
    B.first[count] = total;
    const DeviceInfo &D = device_info();
    if (D.device < 0) return EMDQ_ECUDA;
    int nmax = 0;
    for (int b = 0; b < count; ++b) nmax = n[b] > nmax ? n[b] : nmax;
    if (nmax <= kGridMaxN) {
        static int attr_set = -1;
        if (attr_set != D.device) {
            if (cudaFuncSetAttribute(warm_start_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)grid_layout(kGridMaxN).total) != cudaSuccess)
                return EMDQ_ECUDA;
            attr_set = D.device;
        }
        WarmGridBatch G;
        G.count = count;
        G.nmax = nmax;
        // kGridQueries matches per block; a launch too small to give every SM a block (one
        // frame, a few pairs) takes fewer per block, down to one per warp, so that its
        // latency is not set by a few blocks walking many matches each (each block stages its
        // problem's matches: more blocks repeat that work, which large launches avoid)
        int q = kGridQueries;
        while (q > kNetThreads / 32 && (total + q - 1) / q < D.sms) q >>= 1;
        G.queries = q;
        int blocks = 0;
        for (int b = 0; b < count; ++b) {
            G.src[b] = B.src[b];
            G.dst[b] = B.dst[b];
            G.p0[b] = B.p0[b];
            G.n[b] = B.n[b];
            G.block0[b] = blocks;
            blocks += (n[b] + q - 1) / q;
        }
        G.block0[count] = blocks;
        warm_start_grid_kernel<<<blocks, kNetThreads, grid_layout(nmax).total,
                                 static_cast<cudaStream_t>(stream)>>>(G, params);
        return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
    }
    const int want = (total + 7) / 8, cap = 4 * (D.sms > 0 ? D.sms : 152);
    warm_start_batch_kernel<<<want < cap ? want : cap, kNetThreads, 0,
                              static_cast<cudaStream_t>(stream)>>>(B, params);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

extern "C" size_t emdq_mlp_train_workspace_size(int batch)
{
    if (batch < 1) return 0;
    const size_t tiles = (batch + kMlpThreads - 1) / kMlpThreads;
    return align_up(tiles * (kNParams + 1) * sizeof(float), 256);
}

extern "C" emdq_status emdq_mlp_train_step(const float *feat, const float *label, int batch,
                                           float *params, float *adam_m, float *adam_v, int step,
                                           float lr, float *grad_out, float *loss_out,
                                           void *workspace, size_t workspace_bytes, void *stream)
{
    const bool update = step > 0;
    if (!feat || !label || !params || batch < 1 || (update && (!adam_m || !adam_v)) ||
        !(lr >= 0.f))
        return EMDQ_EINVAL;
    const size_t need = emdq_mlp_train_workspace_size(batch);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return EMDQ_EWORKSPACE;
    static int attr_set = -1;
    const DeviceInfo &D = device_info();
    if (D.device < 0) return EMDQ_ECUDA;
    if (attr_set != D.device) {
        if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kGradSmem) != cudaSuccess)
            return EMDQ_ECUDA;
        attr_set = D.device;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int tiles = (batch + kMlpThreads - 1) / kMlpThreads;
    float *partial = static_cast<float *>(workspace);
    mlp_grad_kernel<<<tiles, kMlpThreads, kGradSmem, st>>>(feat, label, batch, params, partial);
    mlp_adam_kernel<<<(kNParams + 1 + 255) / 256, 256, 0, st>>>(
        partial, tiles, batch, params, adam_m, adam_v, grad_out, loss_out, update ? step : 1, lr,
        0.9f, 0.999f, 1e-8f, update ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}
