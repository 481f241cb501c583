// ARAP smoothing of the node warps (Sec. III-D, Eqs. 21-22), on the stream without host round
// trips.  Iteration k: the nodes' positions x_t = W^{k-1}(x_0) (W^0 = W_merge); the ARAP warp
// of every node, the weighted similarity fit of Eqs. ARAP1-3 over its neighbours, which is the
// EMDQ M-step with p = 1 (emdq_fit with no EM iteration: its step 0); the update of Eq. 22,
// W^k = (W_merge + lambda W_ARAP) / (1 + lambda), lambda = (1 + sigma^2) / (1 + 100); the cost
// of Eq. 21 summed over the nodes.  A device flag stops the iterations once the cost rises
// (the previous warps are kept); later launches of the loop then do nothing.
#include <cmath>

#include "common.cuh"

namespace emdq {

constexpr float kSigma2Arap = 100.f;   // Sec. III-D: the fixed uncertainty of the ARAP term
constexpr int kArapThreads = 1024;

struct ArapState {
    float prev;      // cost of the last accepted iteration
    int done;        // the cost rose: the warps are final
};

__device__ __forceinline__ float2 apply_row(const float *w, float x, float y)
{
    const float nr = rsqrtf(w[0] * w[0] + w[1] * w[1]);
    const float c = w[0] * nr, s = w[1] * nr, dx = w[2] * nr, dy = w[3] * nr;
    const float tx = 2.f * (dx * c - dy * s), ty = 2.f * (dx * s + dy * c);
    const float ct = c * c - s * s, st = 2.f * c * s;
    return make_float2(w[4] * (ct * x - st * y + tx), w[4] * (st * x + ct * y + ty));
}

// weighted average of two warp rows: DQ parts (each normalised by its real part) averaged and
// normalised again, scales averaged
__device__ __forceinline__ void average_rows(const float *a, float wa, const float *b, float wb,
                                             float *out)
{
    const float na = rsqrtf(a[0] * a[0] + a[1] * a[1]), nb = rsqrtf(b[0] * b[0] + b[1] * b[1]);
    float q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = wa * a[k] * na + wb * b[k] * nb;
    const float nq = rsqrtf(q[0] * q[0] + q[1] * q[1]);
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = q[k] * nq;
    out[4] = (wa * a[4] + wb * b[4]) / (wa + wb);
    out[5] = 1.f;
    out[6] = 0.f;
    out[7] = 0.f;
}

__global__ void arap_init_kernel(ArapState *st)
{
    st->prev = INFINITY;
    st->done = 0;
}

__global__ void arap_positions_kernel(const float2 *__restrict__ x0, const float *__restrict__ w,
                                      int nn, const ArapState *__restrict__ st,
                                      float2 *__restrict__ xt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn || st->done) return;
    xt[i] = apply_row(w + 8 * (size_t)i, x0[i].x, x0[i].y);
}

// one block: the Eq. 22 candidates, the Eq. 21 cost in a fixed summation order, the decision,
// then (if accepted) the candidates written over the current warps
__global__ void __launch_bounds__(kArapThreads) arap_update_kernel(
    const float2 *__restrict__ x0, const float *__restrict__ w_merge, const float *__restrict__ s2,
    const float *__restrict__ w_arap, int nn, ArapState *st, float *__restrict__ w_out)
{
    __shared__ float red[kArapThreads / 32];
    __shared__ int accept;
    if (st->done) return;
    float cost = 0.f;
    for (int i = threadIdx.x; i < nn; i += kArapThreads) {
        const float lam = (1.f + s2[i]) / (1.f + kSigma2Arap);
        float cand[8];
        average_rows(w_merge + 8 * (size_t)i, 1.f, w_arap + 8 * (size_t)i, lam, cand);
        const float2 x = x0[i];
        const float2 pm = apply_row(w_merge + 8 * (size_t)i, x.x, x.y);
        const float2 pa = apply_row(w_arap + 8 * (size_t)i, x.x, x.y);
        const float2 pk = apply_row(cand, x.x, x.y);
        const float mx = pm.x - pk.x, my = pm.y - pk.y, ax = pa.x - pk.x, ay = pa.y - pk.y;
        cost += mx * mx + my * my + lam * (ax * ax + ay * ay);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cost += __shfl_xor_sync(0xffffffffu, cost, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cost;
    __syncthreads();
    if (threadIdx.x == 0) {
        float total = 0.f;
        for (int k = 0; k < kArapThreads / 32; ++k) total += red[k];
        accept = !(total > st->prev);
        if (accept) st->prev = total;
        else st->done = 1;
    }
    __syncthreads();
    if (!accept) return;
    for (int i = threadIdx.x; i < nn; i += kArapThreads) {
        const float lam = (1.f + s2[i]) / (1.f + kSigma2Arap);
        average_rows(w_merge + 8 * (size_t)i, 1.f, w_arap + 8 * (size_t)i, lam, w_out + 8 * (size_t)i);
    }
}

struct ArapLayout {
    size_t xt, warap, c, info, state, fit, total;
};

ArapLayout arap_layout(int nn)
{
    auto al = [](size_t v) { return emdq_host::align_up(v, 256); };
    ArapLayout L;
    L.xt = 0;
    L.warap = L.xt + al(sizeof(float2) * (size_t)nn);
    L.c = L.warap + al(sizeof(float) * 8 * (size_t)nn);
    L.info = L.c + al(sizeof(float) * (size_t)nn);
    L.state = L.info + 256;
    L.fit = L.state + 256;
    L.total = L.fit + al(emdq_fit_workspace_size(nn));
    return L;
}

}  // namespace emdq

using namespace emdq;
using namespace emdq_host;

extern "C" size_t emdq_arap_workspace_size(int nn)
{
    if (nn < 3 || nn > emdq_fit_max_n()) return 0;
    return arap_layout(nn).total;
}

extern "C" emdq_status emdq_arap_smooth(const float *x0, const float *w_merge, const float *s2,
                                        int nn, float alpha, int max_iters, float *w_out,
                                        void *workspace, size_t workspace_bytes, void *stream)
{
    if (!x0 || !w_merge || !s2 || !w_out || nn < 3 || max_iters < 0 || !(alpha > 0.f) ||
        !std::isfinite(alpha) || !aligned(x0, 8) || !aligned(w_out, 16))
        return EMDQ_EINVAL;
    if (nn > emdq_fit_max_n()) return EMDQ_ENOTSUP;
    const ArapLayout L = arap_layout(nn);
    if (!workspace || workspace_bytes < L.total || !aligned(workspace, 256)) return EMDQ_EWORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    auto *xt = reinterpret_cast<float2 *>(ws + L.xt);
    auto *wa = reinterpret_cast<float *>(ws + L.warap);
    auto *c = reinterpret_cast<float *>(ws + L.c);
    auto *info = reinterpret_cast<emdq_fit_info *>(ws + L.info);
    auto *state = reinterpret_cast<ArapState *>(ws + L.state);
    if (cudaMemcpyAsync(w_out, w_merge, sizeof(float) * 8 * (size_t)nn, cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess)
        return EMDQ_ECUDA;
    arap_init_kernel<<<1, 1, 0, st>>>(state);
    emdq_params P;
    emdq_default_params(&P);
    P.alpha = alpha;
    P.max_iters = 0;            // step 0 only: the M-step with p = 1
    const auto *x0f = reinterpret_cast<const float2 *>(x0);
    for (int k = 0; k < max_iters; ++k) {
        arap_positions_kernel<<<(nn + 255) / 256, 256, 0, st>>>(x0f, w_out, nn, state, xt);
        const emdq_status rc = emdq_fit(x0, reinterpret_cast<const float *>(xt), nn, 1, 1, &P, nullptr,
                                        wa, c, nullptr, info, ws + L.fit, L.total - L.fit, stream);
        if (rc != EMDQ_OK) return rc;
        arap_update_kernel<<<1, kArapThreads, 0, st>>>(x0f, w_merge, s2, wa, nn, state, w_out);
    }
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}
