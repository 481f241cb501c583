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
// One warp per match.  Each lane keeps the 8 nearest of its candidates i = lane + 32 t,
// sorted by (distance, index); 8 rounds of a warp-wide lexicographic arg-min then pop the
// overall 8 nearest in order -- the same set and order as a full sort.  All lanes end with
// the 16 features.
__device__ __forceinline__ void knn_features_warp(const float2 *__restrict__ src,
                                                  const float2 *__restrict__ dst, int n, int j,
                                                  int lane, float (&f)[2 * kKnn])
{
    const float2 xj = src[j];
    float bd[kKnn];
    int bi[kKnn];
#pragma unroll
    for (int k = 0; k < kKnn; ++k) {
        bd[k] = INFINITY;
        bi[k] = 0x7fffffff;
    }
    for (int i = lane; i < n; i += 32) {
        if (i == j) continue;
        const float2 xi = src[i];
        // float32, one rounding per operation (the same decision as the oracle's)
        const float dx = __fsub_rn(xi.x, xj.x), dy = __fsub_rn(xi.y, xj.y);
        const float d = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        if (d < bd[kKnn - 1] || (d == bd[kKnn - 1] && i < bi[kKnn - 1])) {
            float cd = d;
            int ci = i;
#pragma unroll
            for (int s = 0; s < kKnn; ++s) {
                const bool lt = cd < bd[s] || (cd == bd[s] && ci < bi[s]);
                const float td = bd[s];
                const int ti = bi[s];
                if (lt) {
                    bd[s] = cd;
                    bi[s] = ci;
                    cd = td;
                    ci = ti;
                }
            }
        }
    }
    float nd[kKnn];
    int ni[kKnn];
#pragma unroll
    for (int r = 0; r < kKnn; ++r) {
        float cd = bd[0];
        int ci = bi[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float od = __shfl_xor_sync(0xffffffffu, cd, o);
            const int oi = __shfl_xor_sync(0xffffffffu, ci, o);
            if (od < cd || (od == cd && oi < ci)) {
                cd = od;
                ci = oi;
            }
        }
        nd[r] = cd;
        ni[r] = ci;
        if (bi[0] == ci) {          // this lane held the winner: pop its head
#pragma unroll
            for (int s = 0; s + 1 < kKnn; ++s) {
                bd[s] = bd[s + 1];
                bi[s] = bi[s + 1];
            }
            bd[kKnn - 1] = INFINITY;
            bi[kKnn - 1] = 0x7fffffff;
        }
    }
    // lane k < 8: the residual of neighbour k under the translation match j implies
    const float2 yj = dst[j];
    const float djx = yj.x - xj.x, djy = yj.y - xj.y;
    float mine = 0.f;
    if (lane < kKnn) {
        int idx = ni[0];
#pragma unroll
        for (int k = 1; k < kKnn; ++k)
            if (lane == k) idx = ni[k];
        const float2 xk = src[idx], yk = dst[idx];
        mine = log1pf(hypotf((yk.x - xk.x) - djx, (yk.y - xk.y) - djy));
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
#pragma unroll
    for (int k = 0; k < kKnn; ++k) {
        f[k] = f1[k];
        f[kKnn + k] = log1pf(sqrtf(nd[k]));      // distances, already ascending
    }
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
// Parameters rounded to BF16, staged in shared memory as floats, with W1 and W2 transposed
// ([in][out]) so that lane-per-output reads are conflict-free.
constexpr int kSwW1T = 0, kSwB1 = kSwW1T + kNin * kNh, kSwW2T = kSwB1 + kNh,
              kSwB2 = kSwW2T + kNh * kNh, kSwW3 = kSwB2 + kNh, kSwB3 = kSwW3 + kNh;

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
        if (k < kOffB1) d = kSwW1T + (k % kNin) * kNh + k / kNin;                  // W1[o][m]
        else if (k < kOffW2) d = kSwB1 + (k - kOffB1);
        else if (k < kOffB2) d = kSwW2T + ((k - kOffW2) % kNh) * kNh + (k - kOffW2) / kNh;
        else if (k < kOffW3) d = kSwB2 + (k - kOffB2);
        else if (k < kOffB3) d = kSwW3 + (k - kOffW3);
        else d = kSwB3;
        sw[d] = v;
    }
    __syncthreads();
}

// One sample per warp: lane l computes hidden units l and l + 32 of both layers; inputs
// rounded to BF16, FP32 accumulation; returns the logit z in every lane.
__device__ __forceinline__ float mlp_forward_warp(const float *sw, const float (&f)[2 * kKnn],
                                                  int lane)
{
    float x[kNin];
#pragma unroll
    for (int m = 0; m < kNin; ++m) x[m] = bf(f[m]);
    float a0 = sw[kSwB1 + lane], a1 = sw[kSwB1 + lane + 32];
#pragma unroll
    for (int m = 0; m < kNin; ++m) {
        a0 = fmaf(sw[kSwW1T + m * kNh + lane], x[m], a0);
        a1 = fmaf(sw[kSwW1T + m * kNh + lane + 32], x[m], a1);
    }
    const float h0 = bf(fmaxf(a0, 0.f)), h1 = bf(fmaxf(a1, 0.f));
    float c0 = sw[kSwB2 + lane], c1 = sw[kSwB2 + lane + 32];
#pragma unroll
    for (int k = 0; k < kNh; ++k) {
        const float hk = __shfl_sync(0xffffffffu, k < 32 ? h0 : h1, k & 31);
        c0 = fmaf(sw[kSwW2T + k * kNh + lane], hk, c0);
        c1 = fmaf(sw[kSwW2T + k * kNh + lane + 32], hk, c1);
    }
    float z = sw[kSwW3 + lane] * bf(fmaxf(c0, 0.f)) + sw[kSwW3 + lane + 32] * bf(fmaxf(c1, 0.f));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    return z + sw[kSwB3];
}

constexpr int kNetThreads = 256;
constexpr int kNetSmem = kNParams * sizeof(float);

__global__ void __launch_bounds__(kNetThreads) warm_infer_kernel(const float *__restrict__ feat,
                                                                 int n, const float *__restrict__ w,
                                                                 float *__restrict__ p0)
{
    __shared__ float sw[kNParams];
    stage_params_t(w, sw);
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += nw) {
        float f[2 * kKnn];
#pragma unroll
        for (int m = 0; m < 2 * kKnn; ++m) f[m] = feat[16 * (size_t)j + m];
        const float z = mlp_forward_warp(sw, f, lane);
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
    __shared__ float sw[kNParams];
    stage_params_t(w, sw);
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int total = B.first[B.count];
    int b = 0;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < total; g += nw) {
        while (g >= B.first[b + 1]) ++b;       // g only grows
        const int j = g - B.first[b];
        float f[2 * kKnn];
        knn_features_warp(B.src[b], B.dst[b], B.n[b], j, lane, f);
        const float z = mlp_forward_warp(sw, f, lane);
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
