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

constexpr int kFeatThreads = 64;
constexpr int kFeatChunk = 1024;
constexpr int kMlpThreads = 128;      // also the samples of one training tile

__device__ __forceinline__ float bf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// ------------------------------------------------------------------ features ----------
// Features of match j (valid) of one problem; every thread of the block must call this (the
// candidate positions are staged through shared memory sx, kFeatChunk entries).
__device__ __forceinline__ void knn_features(const float2 *__restrict__ src,
                                             const float2 *__restrict__ dst, int n, int j,
                                             bool valid, float2 *sx, float (&f)[2 * kKnn])
{
    const float2 xj = valid ? src[j] : make_float2(0.f, 0.f);
    float bd[kKnn];
    int bi[kKnn];
#pragma unroll
    for (int k = 0; k < kKnn; ++k) {
        bd[k] = INFINITY;
        bi[k] = 0x7fffffff;
    }
    for (int base = 0; base < n; base += kFeatChunk) {
        const int m = min(kFeatChunk, n - base);
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += blockDim.x) sx[k] = src[base + k];
        __syncthreads();
        if (!valid) continue;
#pragma unroll 4
        for (int k = 0; k < m; ++k) {
            const int i = base + k;
            if (i == j) continue;
            // float32, one rounding per operation (the same decision as the oracle's)
            const float dx = __fsub_rn(sx[k].x, xj.x), dy = __fsub_rn(sx[k].y, xj.y);
            const float d = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            if (d < bd[kKnn - 1] || (d == bd[kKnn - 1] && i < bi[kKnn - 1])) {
                // insert into the sorted list (by distance, then index)
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
    }
    if (!valid) return;
    const float2 yj = dst[j];
    const float djx = yj.x - xj.x, djy = yj.y - xj.y;
    float f1[kKnn];
#pragma unroll
    for (int k = 0; k < kKnn; ++k) {
        const int i = bi[k];
        const float2 xk = src[i], yk = dst[i];
        f1[k] = log1pf(hypotf((yk.x - xk.x) - djx, (yk.y - xk.y) - djy));
        f[kKnn + k] = log1pf(sqrtf(bd[k]));      // already ascending
    }
    // sort the residuals ascending (odd-even transposition, fixed network)
#pragma unroll
    for (int r = 0; r < kKnn; ++r)
#pragma unroll
        for (int k = r & 1; k + 1 < kKnn; k += 2) {
            const float lo = fminf(f1[k], f1[k + 1]), hi = fmaxf(f1[k], f1[k + 1]);
            f1[k] = lo;
            f1[k + 1] = hi;
        }
#pragma unroll
    for (int k = 0; k < kKnn; ++k) f[k] = f1[k];
}

__global__ void __launch_bounds__(kFeatThreads) warm_features_kernel(
    const float2 *__restrict__ src, const float2 *__restrict__ dst, int n,
    float *__restrict__ feat)
{
    __shared__ float2 sx[kFeatChunk];
    const int j = blockIdx.x * kFeatThreads + threadIdx.x;
    float f[2 * kKnn];
    knn_features(src, dst, n, j, j < n, sx, f);
    if (j >= n) return;
    float4 *o = reinterpret_cast<float4 *>(feat + 16 * (size_t)j);
    o[0] = make_float4(f[0], f[1], f[2], f[3]);
    o[1] = make_float4(f[4], f[5], f[6], f[7]);
    o[2] = make_float4(f[8], f[9], f[10], f[11]);
    o[3] = make_float4(f[12], f[13], f[14], f[15]);
}

// ------------------------------------------------------------------ network ------------
// Parameters rounded to BF16, staged in shared memory as floats.
__device__ __forceinline__ void stage_params(const float *__restrict__ w, float *sw)
{
    for (int k = threadIdx.x; k < kNParams; k += blockDim.x) sw[k] = bf(w[k]);
    __syncthreads();
}

// Forward of one sample from its BF16-rounded input: h1, h2 (post-ReLU, rounded to
// BF16), FP32 accumulation; returns the logit z.
__device__ __forceinline__ float mlp_forward(const float *sw, const float (&x)[kNin],
                                             float (&h1)[kNh])
{
#pragma unroll
    for (int o = 0; o < kNh; ++o) {
        float acc = sw[kOffB1 + o];
#pragma unroll
        for (int m = 0; m < kNin; ++m) acc = fmaf(sw[kOffW1 + o * kNin + m], x[m], acc);
        h1[o] = bf(fmaxf(acc, 0.f));
    }
    // second layer: 8 outputs at a time (8 independent accumulation chains)
    float z = sw[kOffB3];
#pragma unroll 1
    for (int o0 = 0; o0 < kNh; o0 += 8) {
        float acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = sw[kOffB2 + o0 + u];
#pragma unroll
        for (int k = 0; k < kNh; ++k)
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = fmaf(sw[kOffW2 + (o0 + u) * kNh + k], h1[k], acc[u]);
#pragma unroll
        for (int u = 0; u < 8; ++u) z = fmaf(sw[kOffW3 + o0 + u], bf(fmaxf(acc[u], 0.f)), z);
    }
    return z;
}

__global__ void __launch_bounds__(kMlpThreads) warm_infer_kernel(const float *__restrict__ feat,
                                                                 int n, const float *__restrict__ w,
                                                                 float *__restrict__ p0)
{
    __shared__ float sw[kNParams];
    stage_params(w, sw);
    const int j = blockIdx.x * kMlpThreads + threadIdx.x;
    if (j >= n) return;
    float x[kNin], h1[kNh];
#pragma unroll
    for (int m = 0; m < kNin; ++m) x[m] = bf(feat[16 * (size_t)j + m]);
    const float z = mlp_forward(sw, x, h1);
    p0[j] = 1.f / (1.f + expf(-z));
}

// Features + network for many problems in one launch: block -> (problem, 128 matches).
constexpr int kWarmBatchMax = 64;
struct WarmBatch {
    const float2 *src[kWarmBatchMax];
    const float2 *dst[kWarmBatchMax];
    float *p0[kWarmBatchMax];
    int n[kWarmBatchMax];
    int first_block[kWarmBatchMax + 1];     // prefix sums of the problems' block counts
    int count;
};

__global__ void __launch_bounds__(kFeatThreads) warm_start_batch_kernel(
    const __grid_constant__ WarmBatch B, const float *__restrict__ w)
{
    __shared__ float sw[kNParams];
    __shared__ float2 sx[kFeatChunk];
    int b = 0;
    while (b + 1 < B.count && (int)blockIdx.x >= B.first_block[b + 1]) ++b;
    const int j = (blockIdx.x - B.first_block[b]) * kFeatThreads + threadIdx.x;
    const int n = B.n[b];
    stage_params(w, sw);
    float f[2 * kKnn];
    knn_features(B.src[b], B.dst[b], n, j, j < n, sx, f);
    if (j >= n) return;
    float x[kNin], h1[kNh];
#pragma unroll
    for (int m = 0; m < kNin; ++m) x[m] = bf(f[m]);
    const float z = mlp_forward(sw, x, h1);
    B.p0[b][j] = 1.f / (1.f + expf(-z));
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
    warm_features_kernel<<<(n + kFeatThreads - 1) / kFeatThreads, kFeatThreads, 0,
                           static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float2 *>(src), reinterpret_cast<const float2 *>(dst), n, feat_out);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

extern "C" emdq_status emdq_warm_infer(const float *feat, int n, const float *params,
                                       float *p0_out, void *stream)
{
    if (!feat || !params || !p0_out || n < 1) return EMDQ_EINVAL;
    warm_infer_kernel<<<(n + kMlpThreads - 1) / kMlpThreads, kMlpThreads, 0,
                        static_cast<cudaStream_t>(stream)>>>(feat, n, params, p0_out);
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
    int blocks = 0;
    for (int b = 0; b < count; ++b) {
        if (!src[b] || !dst[b] || !p0_out[b] || n[b] < kKnn + 1) return EMDQ_EINVAL;
        if (!aligned(src[b], 8) || !aligned(dst[b], 8)) return EMDQ_EINVAL;
        B.src[b] = reinterpret_cast<const float2 *>(src[b]);
        B.dst[b] = reinterpret_cast<const float2 *>(dst[b]);
        B.p0[b] = p0_out[b];
        B.n[b] = n[b];
        B.first_block[b] = blocks;
        blocks += (n[b] + kFeatThreads - 1) / kFeatThreads;
    }
    B.first_block[count] = blocks;
    warm_start_batch_kernel<<<blocks, kFeatThreads, 0, static_cast<cudaStream_t>(stream)>>>(B, params);
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
