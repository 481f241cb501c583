// EMDQ fit on the GPU: one cooperative, persistent launch runs step 0 and every EM
// iteration, synchronising its CTAs with bounded grid barriers, so that a whole fit costs
// one launch and no host round trip.
//
// Work split per iteration (N matches, G CTAs of 8 warps, one warp per match row):
//   E-step      every CTA computes all N posteriors redundantly into shared memory
//               (identical inputs and reduction order, hence identical convergence
//               decisions in every CTA without an extra barrier)
//   M-step      warp w fits rows i = w, w + 8G, ...  The weighted similarity fit needs
//               the centred second moments of Eqs. 18-19; accumulating raw moments and
//               centring afterwards cancels catastrophically (it is why an FP64 finish
//               would be needed).  Instead two passes over j: the weighted centroid,
//               then the moments about it, so nothing cancels and FP32 products and sums
//               suffice (local coordinates x_j - x_i, y_j - y_i keep the values small).
//   barrier
//   residuals   warp w computes the leave-one-out blend at x_j for its rows j, the blend
//               taken relative to row j's own warp (exact: the blend is linear) to keep
//               the FP32 sums small                                 -> e_j (global)
//   barrier
//   sigma^2, gamma from the per-CTA partial sums, in a fixed order.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace emdq {

constexpr int kFitThreads = 256;
constexpr int kFitWarps = kFitThreads / 32;
constexpr int kFitMaxN = 5120;         // shared memory: 40 bytes per match
constexpr int kFitMaxGrid = 1024;
constexpr int kFitEPerThread = (kFitMaxN + kFitThreads - 1) / kFitThreads;   // residuals per thread

struct FitArgs {
    const float2 *src;
    const float2 *dst;
    int n;
    float alpha2;        // alpha * log2(e): weights are exp2(-alpha2 d^2)
    float inv_area;
    int max_iters;
    float tol;
    float sigma2_floor;
    const float *p0;
    float *q_out;
    float *c_out;
    float *p_out;
    emdq_fit_info *info;
    float *e;            // n residuals^2 (workspace)
    float4 *cen;         // n weighted centroids of the last M-step, local coordinates (workspace)
    float *partials;     // one float2 partial sum per CTA of the group (workspace)
    unsigned *bar;       // barrier arrival counter, zero at launch (workspace)
    int *flag;           // device status, zero at launch (workspace)
};

struct FitSmem {
    float2 *x, *y;
    float *p;
    float *qa, *qb, *qu, *qv, *qs;   // warp rows, SoA
};

__device__ __forceinline__ FitSmem fit_smem(int n)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FitSmem s;
    s.x = reinterpret_cast<float2 *>(smem_raw);
    s.y = s.x + n;
    s.p = reinterpret_cast<float *>(s.y + n);
    s.qa = s.p + n;
    s.qb = s.qa + n;
    s.qu = s.qb + n;
    s.qv = s.qu + n;
    s.qs = s.qv + n;
    return s;
}

// Grid-wide barrier with a bounded wait.  `epoch` counts barriers passed (same in every
// CTA).  Returns false if this CTA gave up waiting (the status flag is then ETIMEOUT).
__device__ bool grid_barrier(unsigned *bar, int *flag, unsigned &epoch, int ncta)
{
    __shared__ int timed_out;
    __syncthreads();
    epoch += 1;
    if (threadIdx.x == 0) {
        timed_out = 0;
        const unsigned target = epoch * static_cast<unsigned>(ncta);
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        unsigned spins = 0;
        while (ld_acquire_gpu(bar) < target) {
            if (++spins > kSpinLimit) {
                raise_status(flag, EMDQ_ETIMEOUT);
                timed_out = 1;
                break;
            }
            if (spins > 2048) __nanosleep(64);   // poll hot first, then back off
        }
        __threadfence();
    }
    __syncthreads();
    return !timed_out;
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Eqs. 18-20 from the weight W, the weighted centroids (local coordinates) and the centred
// moments: rotation (2-D closed form), scale (norm ratio), translation.  Lane 0 writes the
// q row and the centroid.
__device__ __forceinline__ void mstep_finish(const FitArgs &A, int i, float2 xi, float2 yi,
                                             float W, float ab0, float ab1, float bb0, float bb1,
                                             float vx, float vy, float c00, float c01, float c10,
                                             float c11, int lane)
{
    // Eq. 18 in 2-D: the rotation angle th maximising tr(R^T C_t C_0^T) has direction
    // (a, b) = (c00 + c11, c10 - c01); its half angle (the DQ real part) is the direction
    // of (rho + a, b), or of (b, rho - a) when a < 0 (no cancellation).
    const float a = c00 + c11, b = c10 - c01;
    const float rho = hypotf(a, b);
    float h0, h1;
    if (a >= 0.f) { h0 = rho + a; h1 = b; }
    else if (b >= 0.f) { h0 = b; h1 = rho - a; }
    else { h0 = -b; h1 = a - rho; }
    const float hn = hypotf(h0, h1);
    float c = 1.f, sn = 0.f;
    if (hn > 0.f) { c = h0 / hn; sn = h1 / hn; }
    // Eq. 19: norm ratio
    const float sc = sqrtf(vy / vx);
    // Eq. 20: t = ybar / s - R xbar in global coordinates
    const float ct = c * c - sn * sn, st = 2.f * c * sn;
    const float xg0 = xi.x + ab0, xg1 = xi.y + ab1;
    const float yg0 = yi.x + bb0, yg1 = yi.y + bb1;
    const float tx = yg0 / sc - (ct * xg0 - st * xg1);
    const float ty = yg1 / sc - (st * xg0 + ct * xg1);
    const bool ok = W > 0.f && isfinite(W) && vx > 0.f && isfinite(sc) && isfinite(tx) &&
                    isfinite(ty);
    if (lane != 0) return;
    float row[5] = {1.f, 0.f, 0.f, 0.f, 1.f};
    if (ok) {
        row[0] = c;
        row[1] = sn;
        row[2] = 0.5f * (tx * c + ty * sn);
        row[3] = 0.5f * (ty * c - tx * sn);
        row[4] = sc;
    } else {
        raise_status(A.flag, EMDQ_EDEGENERATE);
    }
    float4 *dst = reinterpret_cast<float4 *>(A.q_out + 8 * (size_t)i);
    __stcg(dst, make_float4(row[0], row[1], row[2], row[3]));
    __stcg(dst + 1, make_float4(row[4], 1.f, 0.f, 0.f));
    __stcg(A.cen + i, ok ? make_float4(ab0, ab1, bb0, bb1) : make_float4(0.f, 0.f, 0.f, 0.f));
}

// M-step of row i (one warp): weights om_j = p_j exp(-alpha |x_j - x_i|^2), local
// coordinates a = x_j - x_i, b = y_j - y_i.  The similarity fit needs the moments about
// the weighted centroid; summing raw moments and centring afterwards cancels.
//   first round: two passes -- W and the centroid, then the moments about it;
//   later rounds: one pass about the previous round's centroid s of this row (the
//     weights change little from round to round, so the centroid moves by far less than
//     the spread and the final correction W |centroid - s|^2 cancels nothing).
__device__ void mstep_row(const FitArgs &A, const FitSmem &S, int i, int lane, bool first)
{
    const int n = A.n;
    const float2 xi = S.x[i], yi = S.y[i];
    float4 sh = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!first) sh = __ldcg(A.cen + i);
    if (first) {
        float W = 0.f, sa0 = 0.f, sa1 = 0.f, sb0 = 0.f, sb1 = 0.f;
#pragma unroll 4
        for (int j = lane; j < n; j += 32) {
            const float2 xj = S.x[j], yj = S.y[j];
            const float a0 = xj.x - xi.x, a1 = xj.y - xi.y;
            const float om = S.p[j] * ex2_ftz(-A.alpha2 * (a0 * a0 + a1 * a1));
            W += om;
            sa0 += om * a0;
            sa1 += om * a1;
            sb0 += om * (yj.x - yi.x);
            sb1 += om * (yj.y - yi.y);
        }
        W = warp_sum_f(W);
        sa0 = warp_sum_f(sa0);
        sa1 = warp_sum_f(sa1);
        sb0 = warp_sum_f(sb0);
        sb1 = warp_sum_f(sb1);
        if (W > 0.f && isfinite(W)) sh = make_float4(sa0 / W, sa1 / W, sb0 / W, sb1 / W);
    }
    // one pass about the shift sh: W, first moments (for the small correction) and the
    // second moments
    float W = 0.f, su0 = 0.f, su1 = 0.f, sv0 = 0.f, sv1 = 0.f;
    float vx = 0.f, vy = 0.f, c00 = 0.f, c01 = 0.f, c10 = 0.f, c11 = 0.f;
#pragma unroll 4
    for (int j = lane; j < n; j += 32) {
        const float2 xj = S.x[j], yj = S.y[j];
        const float a0 = xj.x - xi.x, a1 = xj.y - xi.y;
        const float om = S.p[j] * ex2_ftz(-A.alpha2 * (a0 * a0 + a1 * a1));
        const float u0 = a0 - sh.x, u1 = a1 - sh.y;
        const float v0 = (yj.x - yi.x) - sh.z, v1 = (yj.y - yi.y) - sh.w;
        const float ou0 = om * u0, ou1 = om * u1;
        W += om;
        su0 += ou0;
        su1 += ou1;
        sv0 += om * v0;
        sv1 += om * v1;
        vx += ou0 * u0 + ou1 * u1;          // |vector(C_0)|^2 about the shift
        vy += om * (v0 * v0 + v1 * v1);     // |vector(C_t)|^2 about the shift
        c00 += v0 * ou0;                    // C_t C_0^T about the shift
        c01 += v0 * ou1;
        c10 += v1 * ou0;
        c11 += v1 * ou1;
    }
    W = warp_sum_f(W);
    su0 = warp_sum_f(su0);
    su1 = warp_sum_f(su1);
    sv0 = warp_sum_f(sv0);
    sv1 = warp_sum_f(sv1);
    vx = warp_sum_f(vx);
    vy = warp_sum_f(vy);
    c00 = warp_sum_f(c00);
    c01 = warp_sum_f(c01);
    c10 = warp_sum_f(c10);
    c11 = warp_sum_f(c11);
    // move the moments from the shift to the centroid: m_c = m_s - W d d'^T, d = mean - sh
    float du0 = 0.f, du1 = 0.f, dv0 = 0.f, dv1 = 0.f;
    if (W > 0.f) {
        du0 = su0 / W;
        du1 = su1 / W;
        dv0 = sv0 / W;
        dv1 = sv1 / W;
    }
    vx -= W * (du0 * du0 + du1 * du1);
    vy -= W * (dv0 * dv0 + dv1 * dv1);
    c00 -= W * dv0 * du0;
    c01 -= W * dv0 * du1;
    c10 -= W * dv1 * du0;
    c11 -= W * dv1 * du1;
    mstep_finish(A, i, xi, yi, W, sh.x + du0, sh.y + du1, sh.z + dv0, sh.w + dv1, vx, vy, c00,
                 c01, c10, c11, lane);
}

// Leave-one-out residual of row j (one warp); returns e_j on lane 0.
__device__ float residual_row(const FitArgs &A, const FitSmem &S, int j, int lane)
{
    const int n = A.n;
    const float2 xj = S.x[j];
    const float ra = S.qa[j], rb = S.qb[j], ru = S.qu[j], rv = S.qv[j], rs = S.qs[j];
    float w0 = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll 4
    for (int i = lane; i < n; i += 32) {
        if (i == j) continue;                         // leave one out
        const float2 xi = S.x[i];
        const float dx = xi.x - xj.x, dy = xi.y - xj.y;
        const float w = S.p[i] * ex2_ftz(-A.alpha2 * (dx * dx + dy * dy));
        w0 += w;
        a0 += w * (S.qa[i] - ra);
        a1 += w * (S.qb[i] - rb);
        a2 += w * (S.qu[i] - ru);
        a3 += w * (S.qv[i] - rv);
        a4 += w * (S.qs[i] - rs);
    }
    w0 = warp_sum_f(w0);
    a0 = warp_sum_f(a0);
    a1 = warp_sum_f(a1);
    a2 = warp_sum_f(a2);
    a3 = warp_sum_f(a3);
    a4 = warp_sum_f(a4);
    if (!(w0 > 0.f)) return INFINITY;
    const float inv = 1.f / w0;
    const float2 yh = apply_blend(ra + a0 * inv, rb + a1 * inv, ru + a2 * inv, rv + a3 * inv,
                                  rs + a4 * inv, xj.x, xj.y);
    const float2 yj = S.y[j];
    const float r0 = yj.x - yh.x, r1 = yj.y - yh.y;
    return r0 * r0 + r1 * r1;
}

// Block-wide sums of two floats in a fixed order: warp butterflies, then every thread
// adds the 8 warp totals in warp order, so every thread (and every CTA, given the same
// inputs) holds the same bits.
__device__ float2 block_sum2(float a, float b, float2 *red)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    a = warp_sum_f(a);
    b = warp_sum_f(b);
    if (lane == 0) red[w] = make_float2(a, b);
    __syncthreads();
    float2 t = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kFitWarps; ++k) {
        t.x += red[k].x;
        t.y += red[k].y;
    }
    __syncthreads();
    return t;
}

// Grid barrier, then the device status word as every thread of every CTA sees it.
__device__ int barrier_status(const FitArgs &A, unsigned &epoch, int *s_flag, int ncta)
{
    const bool ok = grid_barrier(A.bar, A.flag, epoch, ncta);
    if (threadIdx.x == 0) *s_flag = ok ? __ldcg(A.flag) : (int)EMDQ_ETIMEOUT;
    __syncthreads();
    return *s_flag;
}

// One fit on a group of `ncta` co-resident CTAs; `rank` is this CTA's index in the group.
__device__ __forceinline__ void fit_body(const FitArgs &A, int rank, int ncta)
{
    const int n = A.n;
    const FitSmem S = fit_smem(n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gwarp = rank * kFitWarps + warp, nwarps = ncta * kFitWarps;
    __shared__ float2 red[kFitWarps];
    __shared__ int s_flag;
    unsigned epoch = 0;

    // stage the matches and the initial weights; every CTA checks every input
    int bad = 0;
    float p0sum = 0.f;
    for (int j = threadIdx.x; j < n; j += kFitThreads) {
        const float2 x = A.src[j], y = A.dst[j];
        S.x[j] = x;
        S.y[j] = y;
        const float p = A.p0 ? A.p0[j] : 1.f;
        S.p[j] = p;
        p0sum += p;
        bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(y.x) && isfinite(y.y) && isfinite(p));
    }
    bad = __syncthreads_or(bad);
    if (bad) {
        if (rank == 0 && threadIdx.x == 0) {
            A.info->status = EMDQ_ENONFINITE;
            A.info->iters = 0;
        }
        return;
    }
    float gamma = 0.5f;
    if (A.p0) gamma = fminf(fmaxf(block_sum2(p0sum, 0.f, red).x / n, 0.05f), 0.95f);

    // residuals of this CTA's rows and its partial sums, then the barrier
    auto residuals_and_barrier = [&]() -> int {
        for (int i = threadIdx.x; i < n; i += kFitThreads) {
            const float4 r0 = __ldcg(reinterpret_cast<const float4 *>(A.q_out + 8 * (size_t)i));
            const float r4 = __ldcg(A.q_out + 8 * (size_t)i + 4);
            S.qa[i] = r0.x;
            S.qb[i] = r0.y;
            S.qu[i] = r0.z;
            S.qv[i] = r0.w;
            S.qs[i] = r4;
        }
        __syncthreads();
        float pe = 0.f, ps = 0.f;
        for (int j = gwarp; j < n; j += nwarps) {
            const float e = residual_row(A, S, j, lane);
            if (lane == 0) {
                __stcg(A.e + j, e);
                if (isfinite(e)) {
                    pe += S.p[j] * e;
                    ps += S.p[j];
                }
            }
        }
        const float2 t = block_sum2(lane == 0 ? pe : 0.f, lane == 0 ? ps : 0.f, red);
        if (threadIdx.x == 0) __stcg(reinterpret_cast<float2 *>(A.partials) + rank, t);
        return barrier_status(A, epoch, &s_flag, ncta);
    };
    // after that barrier: this thread's residuals (all N are needed by every CTA) and
    // sigma^2 from the per-CTA partials, loads issued together so their latencies overlap;
    // every warp reduces the partials itself, in the same order
    float ev[kFitEPerThread];
    auto load_e_and_sigma2 = [&]() -> float {
#pragma unroll
        for (int k = 0; k < kFitEPerThread; ++k) {
            const int j = threadIdx.x + k * kFitThreads;
            ev[k] = j < n ? __ldcg(A.e + j) : 0.f;
        }
        float num = 0.f, den = 0.f;
        for (int b = lane; b < ncta; b += 32) {
            const float2 v = __ldcg(reinterpret_cast<const float2 *>(A.partials) + b);
            num += v.x;
            den += v.y;
        }
        num = warp_sum_f(num);
        den = warp_sum_f(den);
        const float s2 = den > 0.f ? num / (2.f * den) : A.sigma2_floor;
        return fmaxf(s2, A.sigma2_floor);
    };

    // step 0
    float sigma2 = A.sigma2_floor;
    for (int i = gwarp; i < n; i += nwarps) mstep_row(A, S, i, lane, true);
    int st = barrier_status(A, epoch, &s_flag, ncta);
    if (st < EMDQ_EDEGENERATE) st = residuals_and_barrier();
    if (st < EMDQ_EDEGENERATE) sigma2 = load_e_and_sigma2();

    int it = 0;
    bool converged = false;
    const float two_pi = 6.28318530717958647692f;
    while (st < EMDQ_EDEGENERATE && it < A.max_iters) {
        ++it;
        // E-step: every CTA, all N posteriors
        float dpmax = 0.f, psum = 0.f;
        const float norm = 1.f / (two_pi * sigma2);
        const float outl = (1.f - gamma) * A.inv_area;
#pragma unroll
        for (int k = 0; k < kFitEPerThread; ++k) {
            const int j = threadIdx.x + k * kFitThreads;
            if (j < n) {
                const float e = ev[k];
                const float G = isfinite(e) ? expf(-e / (2.f * sigma2)) * norm : 0.f;
                const float pn = gamma * G / (gamma * G + outl);
                dpmax = fmaxf(dpmax, fabsf(pn - S.p[j]));
                S.p[j] = pn;
                psum += pn;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dpmax = fmaxf(dpmax, __shfl_xor_sync(0xffffffffu, dpmax, o));
        psum = warp_sum_f(psum);
        if (lane == 0) red[warp] = make_float2(dpmax, psum);
        __syncthreads();
        float dpall = 0.f, ptot = 0.f;
#pragma unroll
        for (int k = 0; k < kFitWarps; ++k) {
            dpall = fmaxf(dpall, red[k].x);
            ptot += red[k].y;
        }
        __syncthreads();
        const float gamma_next = fminf(fmaxf(ptot / n, 0.05f), 0.95f);
        // M-step with the new weights, then residuals and sigma^2
        for (int i = gwarp; i < n; i += nwarps) mstep_row(A, S, i, lane, false);
        st = barrier_status(A, epoch, &s_flag, ncta);
        if (st < EMDQ_EDEGENERATE) st = residuals_and_barrier();
        if (st < EMDQ_EDEGENERATE) sigma2 = load_e_and_sigma2();
        gamma = gamma_next;
        if (dpall < A.tol) {
            converged = true;
            break;
        }
    }

    if (rank == 0) {
        for (int j = threadIdx.x; j < n; j += kFitThreads) {
            const float p = S.p[j];
            A.c_out[j] = p >= 0.5f ? p : 0.f;
            if (A.p_out) A.p_out[j] = p;
        }
        if (threadIdx.x == 0) {
            const int f = st >= EMDQ_EDEGENERATE ? st : __ldcg(A.flag);
            int out = EMDQ_OK;
            if (f == EMDQ_ETIMEOUT) out = EMDQ_ETIMEOUT;
            else if (f == EMDQ_EDEGENERATE) out = EMDQ_EDEGENERATE;
            else if (!converged) out = EMDQ_ENOCONV;
            A.info->status = out;
            A.info->iters = it;
            A.info->sigma2 = sigma2;
            A.info->gamma = gamma;
        }
    }
}

__global__ void __launch_bounds__(kFitThreads, 2) emdq_fit_kernel(FitArgs A)
{
    fit_body(A, blockIdx.x, gridDim.x);
}

// Many fits in one cooperative launch: problem b runs on CTAs [b * group, (b + 1) * group),
// with its own barrier counter, status word and partial sums.
constexpr int kFitBatchMax = 64;
struct FitBatch {
    FitArgs a[kFitBatchMax];
};

__global__ void __launch_bounds__(kFitThreads, 2) emdq_fit_batch_kernel(const __grid_constant__ FitBatch B,
                                                                      int group)
{
    const int b = blockIdx.x / group;
    fit_body(B.a[b], blockIdx.x - b * group, group);
}

}  // namespace emdq

using namespace emdq;
using namespace emdq_host;

namespace {
// Fit workspace: residuals e[n], centroids cen[n], per-CTA partial sums, then 256 bytes for
// the barrier counter and the status word.
struct FitLayout {
    size_t e_off, cen_off, part_off, bar_off, total;
};
constexpr size_t al256(size_t v) { return (v + 255) / 256 * 256; }
constexpr FitLayout fit_layout(int n)
{
    return FitLayout{0, al256(sizeof(float) * (size_t)n),
                     al256(sizeof(float) * (size_t)n) + al256(sizeof(float4) * (size_t)n),
                     al256(sizeof(float) * (size_t)n) + al256(sizeof(float4) * (size_t)n) +
                         al256(sizeof(double) * 2 * kFitMaxGrid),
                     al256(sizeof(float) * (size_t)n) + al256(sizeof(float4) * (size_t)n) +
                         al256(sizeof(double) * 2 * kFitMaxGrid) + 256};
}
size_t fit_smem_bytes(int n) { return (size_t)n * 40; }
}  // namespace

extern "C" int emdq_fit_max_n(void) { return kFitMaxN; }

extern "C" size_t emdq_fit_workspace_size(int n)
{
    if (n < 0) return 0;
    return fit_layout(n).total;
}

extern "C" emdq_status emdq_fit(const float *src, const float *dst, int n, int frame_w,
                                int frame_h, const emdq_params *prm, const float *p0,
                                float *q_out, float *c_out, float *p_out, emdq_fit_info *info,
                                void *workspace, size_t workspace_bytes, void *stream)
{
    emdq_params P;
    emdq_default_params(&P);
    if (prm) P = *prm;
    if (!src || !dst || !q_out || !c_out || !info || n < 3 || frame_w < 1 || frame_h < 1 ||
        P.max_iters < 0 || !(P.tol_p >= 0.f) || !(P.sigma2_floor > 0.f))
        return EMDQ_EINVAL;
    if (!aligned(src, 8) || !aligned(dst, 8) || !aligned(q_out, 16) || !aligned(info, 4))
        return EMDQ_EINVAL;
    if (n > kFitMaxN) return EMDQ_ENOTSUP;
    const FitLayout L = fit_layout(n);
    if (!workspace || workspace_bytes < L.total || !aligned(workspace, 256)) return EMDQ_EWORKSPACE;
    const DeviceInfo &D = device_info();
    if (D.device < 0) return EMDQ_ECUDA;
    const size_t smem = fit_smem_bytes(n);
    if (smem > D.smem_optin) return EMDQ_ENOTSUP;

    static std::mutex mu;
    static int attr_set_dev = -1;
    {
        std::lock_guard<std::mutex> g(mu);
        if (attr_set_dev != D.device) {
            if (cudaFuncSetAttribute(emdq_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kFitMaxN * 40)) != cudaSuccess)
                return EMDQ_ECUDA;
            attr_set_dev = D.device;
        }
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, emdq_fit_kernel, kFitThreads, smem) !=
            cudaSuccess || per_sm < 1)
        return EMDQ_ECUDA;
    int grid = (n + kFitWarps - 1) / kFitWarps;
    const int cap = D.sms * per_sm;
    if (grid > cap) grid = cap;
    if (grid > kFitMaxGrid) grid = kFitMaxGrid;

    char *ws = static_cast<char *>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // barrier counter and status flag start at zero
    if (cudaMemsetAsync(ws + L.bar_off, 0, 256, st) != cudaSuccess) return EMDQ_ECUDA;

    FitArgs A;
    A.src = reinterpret_cast<const float2 *>(src);
    A.dst = reinterpret_cast<const float2 *>(dst);
    A.n = n;
    const double alpha = P.alpha > 0.f ? P.alpha : emdq_alpha_for_frame(frame_w, frame_h);
    A.alpha2 = static_cast<float>(alpha * 1.4426950408889634074);
    A.inv_area = 1.f / (static_cast<float>(frame_w) * static_cast<float>(frame_h));
    A.max_iters = P.max_iters;
    A.tol = P.tol_p;
    A.sigma2_floor = P.sigma2_floor;
    A.p0 = p0;
    A.q_out = q_out;
    A.c_out = c_out;
    A.p_out = p_out;
    A.info = info;
    A.e = reinterpret_cast<float *>(ws + L.e_off);
    A.cen = reinterpret_cast<float4 *>(ws + L.cen_off);
    A.partials = reinterpret_cast<float *>(ws + L.part_off);
    A.bar = reinterpret_cast<unsigned *>(ws + L.bar_off);
    A.flag = reinterpret_cast<int *>(ws + L.bar_off + 64);

    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kFitThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, emdq_fit_kernel, A) != cudaSuccess) return EMDQ_ECUDA;
    return EMDQ_OK;
}


// ------------------------------------------------------------------ emdq_fit_batch -----
namespace {
// Batch workspace: one 256-byte header per problem (barrier counter, status word) packed
// first so that a single memset clears them all, then each problem's residuals and
// partial sums.
size_t batch_body_bytes(int n)
{
    return fit_layout(n).bar_off;      // e, cen and partials; the headers are packed first
}
}  // namespace

extern "C" size_t emdq_fit_batch_workspace_size(const emdq_fit_problem *problems, int count)
{
    if (!problems || count < 1 || count > kFitBatchMax) return 0;
    size_t total = 256 * (size_t)count;
    for (int b = 0; b < count; ++b) {
        if (problems[b].n < 0) return 0;
        total += batch_body_bytes(problems[b].n);
    }
    return total;
}

extern "C" emdq_status emdq_fit_batch(const emdq_fit_problem *problems, int count,
                                      const emdq_params *prm, void *workspace,
                                      size_t workspace_bytes, void *stream)
{
    emdq_params P;
    emdq_default_params(&P);
    if (prm) P = *prm;
    if (!problems || count < 1 || P.max_iters < 0 || !(P.tol_p >= 0.f) || !(P.sigma2_floor > 0.f))
        return EMDQ_EINVAL;
    if (count > kFitBatchMax) return EMDQ_ENOTSUP;
    int max_n = 0;
    for (int b = 0; b < count; ++b) {
        const emdq_fit_problem &q = problems[b];
        if (!q.src || !q.dst || !q.q_out || !q.c_out || !q.info || q.n < 3 || q.frame_w < 1 ||
            q.frame_h < 1)
            return EMDQ_EINVAL;
        if (!aligned(q.src, 8) || !aligned(q.dst, 8) || !aligned(q.q_out, 16) || !aligned(q.info, 4))
            return EMDQ_EINVAL;
        if (q.n > kFitMaxN) return EMDQ_ENOTSUP;
        max_n = q.n > max_n ? q.n : max_n;
    }
    const size_t need = emdq_fit_batch_workspace_size(problems, count);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return EMDQ_EWORKSPACE;
    const DeviceInfo &D = device_info();
    if (D.device < 0) return EMDQ_ECUDA;
    const size_t smem = fit_smem_bytes(max_n);
    if (smem > D.smem_optin) return EMDQ_ENOTSUP;
    static std::mutex mu;
    static int attr_set_dev = -1;
    {
        std::lock_guard<std::mutex> g(mu);
        if (attr_set_dev != D.device) {
            if (cudaFuncSetAttribute(emdq_fit_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kFitMaxN * 40)) != cudaSuccess)
                return EMDQ_ECUDA;
            attr_set_dev = D.device;
        }
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, emdq_fit_batch_kernel, kFitThreads,
                                                      smem) != cudaSuccess || per_sm < 1)
        return EMDQ_ECUDA;
    int group = (D.sms * per_sm) / count;
    const int want = (max_n + kFitWarps - 1) / kFitWarps;
    if (group > want) group = want;
    if (group > kFitMaxGrid) group = kFitMaxGrid;
    if (group < 1) return EMDQ_ENOTSUP;    // more problems than co-resident CTAs

    char *ws = static_cast<char *>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ws, 0, 256 * (size_t)count, st) != cudaSuccess) return EMDQ_ECUDA;
    FitBatch B;
    size_t off = 256 * (size_t)count;
    const double two_log2e = 1.4426950408889634074;
    for (int b = 0; b < count; ++b) {
        const emdq_fit_problem &q = problems[b];
        FitArgs &A = B.a[b];
        A.src = reinterpret_cast<const float2 *>(q.src);
        A.dst = reinterpret_cast<const float2 *>(q.dst);
        A.n = q.n;
        const double alpha = P.alpha > 0.f ? P.alpha : emdq_alpha_for_frame(q.frame_w, q.frame_h);
        A.alpha2 = static_cast<float>(alpha * two_log2e);
        A.inv_area = 1.f / (static_cast<float>(q.frame_w) * static_cast<float>(q.frame_h));
        A.max_iters = P.max_iters;
        A.tol = P.tol_p;
        A.sigma2_floor = P.sigma2_floor;
        A.p0 = q.p0;
        A.q_out = q.q_out;
        A.c_out = q.c_out;
        A.p_out = q.p_out;
        A.info = q.info;
        A.bar = reinterpret_cast<unsigned *>(ws + 256 * (size_t)b);
        A.flag = reinterpret_cast<int *>(ws + 256 * (size_t)b + 64);
        const FitLayout L = fit_layout(q.n);
        A.e = reinterpret_cast<float *>(ws + off + L.e_off);
        A.cen = reinterpret_cast<float4 *>(ws + off + L.cen_off);
        A.partials = reinterpret_cast<float *>(ws + off + L.part_off);
        off += batch_body_bytes(q.n);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(group * count);
    cfg.blockDim = dim3(kFitThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, emdq_fit_batch_kernel, B, group) != cudaSuccess) return EMDQ_ECUDA;
    return EMDQ_OK;
}

// ------------------------------------------------------------------ emdq_fit_noalloc ---
// The same fit for callers that must not allocate device memory: its scratch (residuals,
// per-CTA partial sums, barrier counter, status word) lives in one fixed array in this
// library's device memory, sized for the largest fit (kFitMaxN matches), instead of a
// caller workspace.  Every GPU that loads the library holds the array until exit.
namespace {

constexpr size_t kNoAllocScratchBytes = fit_layout(kFitMaxN).total;   // about 118 KB

static __device__ __align__(256) unsigned char g_fit_scratch[kNoAllocScratchBytes];

// Device address of g_fit_scratch on the current device.  In host code the array's name
// is only a host-side stand-in, so the address is asked of the runtime once per device,
// with that device current, and cached.
void *noalloc_scratch()
{
    static std::mutex mu;
    static void *addr[64] = {};
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_fit_scratch) != cudaSuccess || !p) return nullptr;
        addr[dev] = p;
    }
    return addr[dev];
}

}  // namespace

extern "C" emdq_status emdq_fit_noalloc(const float *src, const float *dst, int n, int frame_w,
                                        int frame_h, const emdq_params *prm, const float *p0,
                                        float *q_out, float *c_out, float *p_out,
                                        emdq_fit_info *info, void *stream)
{
    if (n > kFitMaxN) return EMDQ_ENOTSUP;   // beyond the fixed scratch array
    if (fit_layout(n).total > kNoAllocScratchBytes) return EMDQ_ENOTSUP;
    void *ws = noalloc_scratch();
    if (!ws) return EMDQ_ECUDA;
    // emdq_fit clears the barrier counter and status word before its launch
    return emdq_fit(src, dst, n, frame_w, frame_h, prm, p0, q_out, c_out, p_out, info, ws,
                    kNoAllocScratchBytes, stream);
}
