// EMDQ fit on the GPU: one cooperative, persistent launch runs step 0 and every EM
// iteration, synchronising its CTAs with bounded grid barriers, so that a whole fit costs
// one launch and no host round trip.
//
// Work split per iteration (N matches, G CTAs of 8 warps, one warp per match row):
//   E-step      every CTA computes all N posteriors redundantly into shared memory
//               (identical inputs and reduction order, hence identical convergence
//               decisions in every CTA without an extra barrier)
//   M-step      warp w fits rows i = w, w + 8G, ...: FP32 products over j, per-lane FP32
//               partials, cross-lane sums in compensated (two-sum) FP32, then the
//               centring and the closed form of Eqs. 18-20 in FP64 for the CTA's 8 rows
//               at once (one FP64 instruction serves 8 rows: GB300's FP64 pipe is narrow)
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

struct FitArgs {
    const float2 *src;
    const float2 *dst;
    int n;
    float alpha;
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
    double *partials;    // gridDim.x x 2 (workspace)
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
__device__ bool grid_barrier(unsigned *bar, int *flag, unsigned &epoch)
{
    __shared__ int timed_out;
    __syncthreads();
    epoch += 1;
    if (threadIdx.x == 0) {
        timed_out = 0;
        const unsigned target = epoch * gridDim.x;
        __threadfence();
        atomicAdd(bar, 1u);
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

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Error-free sum of two floats (Knuth two-sum): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Cross-lane sum of a float carried as an unevaluated pair hi + lo (every lane ends with
// the same pair: the xor butterfly is symmetric).
__device__ __forceinline__ void warp_sum_ff(float v, float &hi, float &lo)
{
    hi = v;
    lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, oh, s, e);
        e = __fadd_rn(e, __fadd_rn(lo, ol));
        hi = __fadd_rn(s, e);
        lo = __fsub_rn(e, __fsub_rn(hi, s));
    }
}

constexpr int kMoments = 11;

// M-step partial sums of row i (one warp).  Local coordinates a = x_j - x_i,
// b = y_j - y_i keep the products small.  Lane 0 stores the 11 sums as (hi, lo) pairs.
__device__ void mstep_sums(const FitArgs &A, const FitSmem &S, int i, int lane, float *out)
{
    const int n = A.n;
    const float2 xi = S.x[i], yi = S.y[i];
    float m[kMoments];
#pragma unroll
    for (int k = 0; k < kMoments; ++k) m[k] = 0.f;
    for (int j = lane; j < n; j += 32) {
        const float2 xj = S.x[j], yj = S.y[j];
        const float a0 = xj.x - xi.x, a1 = xj.y - xi.y;
        const float b0 = yj.x - yi.x, b1 = yj.y - yi.y;
        const float aa = a0 * a0 + a1 * a1;
        const float om = S.p[j] * expf(-A.alpha * aa);
        m[0] += om;
        m[1] += om * a0;
        m[2] += om * a1;
        m[3] += om * b0;
        m[4] += om * b1;
        m[5] += om * aa;
        m[6] += om * (b0 * b0 + b1 * b1);
        m[7] += om * b0 * a0;
        m[8] += om * b0 * a1;
        m[9] += om * b1 * a0;
        m[10] += om * b1 * a1;
    }
#pragma unroll
    for (int k = 0; k < kMoments; ++k) {
        float hi, lo;
        warp_sum_ff(m[k], hi, lo);
        if (lane == 0) {
            out[k] = hi;
            out[kMoments + k] = lo;
        }
    }
}

// FP64 centring and closed form of row i from its (hi, lo) sums; writes the q row.
__device__ void mstep_finish(const FitArgs &A, const FitSmem &S, int i, const float *in)
{
    double m[kMoments];
#pragma unroll
    for (int k = 0; k < kMoments; ++k)
        m[k] = static_cast<double>(in[k]) + static_cast<double>(in[kMoments + k]);
    const float2 xi = S.x[i], yi = S.y[i];
    float row[5] = {1.f, 0.f, 0.f, 0.f, 1.f};
    const double dW = m[0];
    bool ok = dW > 0.0;
    if (ok) {
        const double iw = 1.0 / dW;
        const double xb0 = m[1] * iw, xb1 = m[2] * iw, yb0 = m[3] * iw, yb1 = m[4] * iw;
        const double vx = m[5] - dW * (xb0 * xb0 + xb1 * xb1);   // |vector(C_0)|^2
        const double vy = m[6] - dW * (yb0 * yb0 + yb1 * yb1);   // |vector(C_t)|^2
        const double S00 = m[7] - dW * yb0 * xb0, S01 = m[8] - dW * yb0 * xb1;
        const double S10 = m[9] - dW * yb1 * xb0, S11 = m[10] - dW * yb1 * xb1;
        // Eq. 18 in 2-D: the rotation angle th maximising tr(R^T S) has direction
        // (S00 + S11, S10 - S01); its half angle (the DQ real part) is the direction of
        // (rho + a, b), or of (b, rho - a) when a < 0 (no cancellation either way).
        const float a = static_cast<float>(S00 + S11), b = static_cast<float>(S10 - S01);
        const float rho = hypotf(a, b);
        float h0, h1;
        if (a >= 0.f) { h0 = rho + a; h1 = b; }
        else if (b >= 0.f) { h0 = b; h1 = rho - a; }
        else { h0 = -b; h1 = a - rho; }
        const float hn = hypotf(h0, h1);
        float c = 1.f, sn = 0.f;
        if (hn > 0.f) { c = h0 / hn; sn = h1 / hn; }
        // Eq. 19: norm ratio
        const float sc = sqrtf(static_cast<float>(vy) / static_cast<float>(vx));
        // Eq. 20: t = ybar / s - R xbar in global coordinates
        const float ct = c * c - sn * sn, st = 2.f * c * sn;
        const float xg0 = xi.x + static_cast<float>(xb0), xg1 = xi.y + static_cast<float>(xb1);
        const float yg0 = yi.x + static_cast<float>(yb0), yg1 = yi.y + static_cast<float>(yb1);
        const float tx = yg0 / sc - (ct * xg0 - st * xg1);
        const float ty = yg1 / sc - (st * xg0 + ct * xg1);
        ok = vx > 0.0 && isfinite(sc) && isfinite(tx) && isfinite(ty);
        if (ok) {
            row[0] = c;
            row[1] = sn;
            row[2] = 0.5f * (tx * c + ty * sn);
            row[3] = 0.5f * (ty * c - tx * sn);
            row[4] = sc;
        }
    }
    if (!ok) raise_status(A.flag, EMDQ_EDEGENERATE);
    float4 *dst = reinterpret_cast<float4 *>(A.q_out + 8 * (size_t)i);
    __stcg(dst, make_float4(row[0], row[1], row[2], row[3]));
    __stcg(dst + 1, make_float4(row[4], 1.f, 0.f, 0.f));
}

// Leave-one-out residual of row j (one warp); returns e_j on lane 0.
__device__ float residual_row(const FitArgs &A, const FitSmem &S, int j, int lane)
{
    const int n = A.n;
    const float2 xj = S.x[j];
    const float ra = S.qa[j], rb = S.qb[j], ru = S.qu[j], rv = S.qv[j], rs = S.qs[j];
    float w0 = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
    for (int i = lane; i < n; i += 32) {
        if (i == j) continue;                         // leave one out
        const float2 xi = S.x[i];
        const float dx = xi.x - xj.x, dy = xi.y - xj.y;
        const float w = S.p[i] * expf(-A.alpha * (dx * dx + dy * dy));
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

// Sum of per-warp doubles in warp order (deterministic); result valid in thread 0.
__device__ double block_sum_ordered(double v, double *red)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kFitWarps; ++k) s += red[k];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(kFitThreads, 1) emdq_fit_kernel(FitArgs A)
{
    const int n = A.n;
    const FitSmem S = fit_smem(n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gwarp = blockIdx.x * kFitWarps + warp, nwarps = gridDim.x * kFitWarps;
    __shared__ double red[kFitWarps];
    __shared__ double bcast[4];
    __shared__ int s_flag;
    unsigned epoch = 0;

    // stage the matches and the initial weights; every CTA checks every input
    int bad = 0;
    double p0sum = 0.0;
    for (int j = threadIdx.x; j < n; j += kFitThreads) {
        const float2 x = A.src[j], y = A.dst[j];
        S.x[j] = x;
        S.y[j] = y;
        const float p = A.p0 ? A.p0[j] : 1.f;
        S.p[j] = p;
        bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(y.x) && isfinite(y.y) && isfinite(p));
    }
    bad = __syncthreads_or(bad);
    if (bad) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            A.info->status = EMDQ_ENONFINITE;
            A.info->iters = 0;
        }
        return;
    }
    float gamma = 0.5f;
    if (A.p0) {
        for (int j = threadIdx.x; j < n; j += kFitThreads) p0sum += S.p[j];
        // per-warp partials then warp-ordered sum: identical in every CTA
        p0sum = warp_sum_d(p0sum);
        const double tot = block_sum_ordered(p0sum, red);
        if (threadIdx.x == 0) bcast[0] = tot;
        __syncthreads();
        gamma = fminf(fmaxf(static_cast<float>(bcast[0] / n), 0.05f), 0.95f);
    }

    __shared__ float msum[kFitWarps][2 * kMoments];
    auto mstep_all = [&]() {
        const int rounds = (n + nwarps - 1) / nwarps;
        for (int r = 0; r < rounds; ++r) {
            const int i = gwarp + r * nwarps;
            if (i < n) mstep_sums(A, S, i, lane, msum[warp]);
            __syncthreads();
            if (warp == 0 && lane < kFitWarps) {
                const int ii = blockIdx.x * kFitWarps + lane + r * nwarps;
                if (ii < n) mstep_finish(A, S, ii, msum[lane]);
            }
            __syncthreads();
        }
    };
    // residuals for this CTA's rows + its partial sums; then barrier; then sigma^2
    auto residuals_and_sigma2 = [&](float &sigma2) -> bool {
        // every CTA needs all q rows in shared memory
        for (int i = threadIdx.x; i < n; i += kFitThreads) {
            const float4 r0 = __ldcg(reinterpret_cast<const float4 *>(A.q_out + 8 * (size_t)i));
            const float4 r1 = __ldcg(reinterpret_cast<const float4 *>(A.q_out + 8 * (size_t)i) + 1);
            S.qa[i] = r0.x;
            S.qb[i] = r0.y;
            S.qu[i] = r0.z;
            S.qv[i] = r0.w;
            S.qs[i] = r1.x;
        }
        __syncthreads();
        double pe = 0.0, ps = 0.0;
        for (int j = gwarp; j < n; j += nwarps) {
            const float e = residual_row(A, S, j, lane);
            if (lane == 0) {
                __stcg(A.e + j, e);
                if (isfinite(e)) {
                    pe += static_cast<double>(S.p[j]) * e;
                    ps += S.p[j];
                }
            }
        }
        const double tpe = block_sum_ordered(pe, red);
        const double tps = block_sum_ordered(ps, red);
        if (threadIdx.x == 0) {
            __stcg(A.partials + 2 * blockIdx.x, tpe);
            __stcg(A.partials + 2 * blockIdx.x + 1, tps);
        }
        if (!grid_barrier(A.bar, A.flag, epoch)) return false;
        if (warp == 0) {
            // lane-strided FP64 partial sums, then the symmetric butterfly: the same
            // value, bit for bit, in every CTA
            double num = 0.0, den = 0.0;
            for (int b = lane; b < (int)gridDim.x; b += 32) {
                num += __ldcg(A.partials + 2 * b);
                den += __ldcg(A.partials + 2 * b + 1);
            }
            num = warp_sum_d(num);
            den = warp_sum_d(den);
            if (lane == 0) {
                const double s2 = den > 0.0 ? num / (2.0 * den) : A.sigma2_floor;
                bcast[1] = s2 > A.sigma2_floor ? s2 : A.sigma2_floor;
                s_flag = __ldcg(A.flag);
            }
        }
        __syncthreads();
        sigma2 = static_cast<float>(bcast[1]);
        return s_flag < EMDQ_EDEGENERATE;
    };

    // step 0
    float sigma2 = A.sigma2_floor;
    mstep_all();
    bool alive = grid_barrier(A.bar, A.flag, epoch);
    if (alive) {
        if (threadIdx.x == 0) s_flag = __ldcg(A.flag);
        __syncthreads();
        alive = s_flag < EMDQ_EDEGENERATE;
    }
    if (alive) alive = residuals_and_sigma2(sigma2);

    int it = 0;
    bool converged = false;
    const float two_pi = 6.28318530717958647692f;
    while (alive && it < A.max_iters) {
        ++it;
        // E-step: every CTA, all N posteriors
        float dpmax = 0.f;
        float psum = 0.f;
        const float norm = 1.f / (two_pi * sigma2);
        const float outl = (1.f - gamma) * A.inv_area;
        for (int j = threadIdx.x; j < n; j += kFitThreads) {
            const float e = __ldcg(A.e + j);
            const float G = isfinite(e) ? expf(-e / (2.f * sigma2)) * norm : 0.f;
            const float pn = gamma * G / (gamma * G + outl);
            dpmax = fmaxf(dpmax, fabsf(pn - S.p[j]));
            S.p[j] = pn;
            psum += pn;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dpmax = fmaxf(dpmax, __shfl_xor_sync(0xffffffffu, dpmax, o));
        psum = warp_sum_f(psum);
        if (lane == 0) red[warp] = dpmax;
        __syncthreads();
        float dpall = 0.f;
        for (int k = 0; k < kFitWarps; ++k) dpall = fmaxf(dpall, static_cast<float>(red[k]));
        __syncthreads();
        const double ptot = block_sum_ordered(static_cast<double>(psum), red);
        if (threadIdx.x == 0) bcast[2] = ptot;
        __syncthreads();
        const float gamma_next =
            fminf(fmaxf(static_cast<float>(bcast[2] / n), 0.05f), 0.95f);
        // M-step with the new weights
        mstep_all();
        alive = grid_barrier(A.bar, A.flag, epoch);
        if (alive) {
            if (threadIdx.x == 0) s_flag = __ldcg(A.flag);
            __syncthreads();
            alive = s_flag < EMDQ_EDEGENERATE;
        }
        if (alive) alive = residuals_and_sigma2(sigma2);
        gamma = gamma_next;
        if (dpall < A.tol) {
            converged = true;
            break;
        }
    }

    if (blockIdx.x == 0) {
        for (int j = threadIdx.x; j < n; j += kFitThreads) {
            const float p = S.p[j];
            A.c_out[j] = p >= 0.5f ? p : 0.f;
            if (A.p_out) A.p_out[j] = p;
        }
        if (threadIdx.x == 0) {
            const int f = __ldcg(A.flag);
            int st = EMDQ_OK;
            if (f == EMDQ_ETIMEOUT) st = EMDQ_ETIMEOUT;
            else if (f == EMDQ_EDEGENERATE) st = EMDQ_EDEGENERATE;
            else if (!converged) st = EMDQ_ENOCONV;
            A.info->status = st;
            A.info->iters = it;
            A.info->sigma2 = sigma2;
            A.info->gamma = gamma;
        }
    }
}

}  // namespace emdq

using namespace emdq;
using namespace emdq_host;

namespace {
struct FitLayout {
    size_t e_off, part_off, bar_off, total;
};
FitLayout fit_layout(int n)
{
    FitLayout L;
    L.e_off = 0;
    L.part_off = align_up(sizeof(float) * (size_t)n, 256);
    L.bar_off = L.part_off + align_up(sizeof(double) * 2 * kFitMaxGrid, 256);
    L.total = L.bar_off + 256;
    return L;
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
    A.alpha = P.alpha > 0.f ? P.alpha : emdq_alpha_for_frame(frame_w, frame_h);
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
    A.partials = reinterpret_cast<double *>(ws + L.part_off);
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
