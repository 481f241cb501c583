// ARAP smoothing of the node warps (Sec. III-D, Eqs. 16-17, ARAP1-3, 21-22), on the stream
// without host round trips.  Iteration k: the nodes' positions x_t = W^{k-1}(x_0)
// (W^0 = W_merge); the ARAP warp of every node from the motion x_j,0 -> x_j,t of all nodes j,
// as printed: node-centred columns w_j^i (x_j - x_i) with the weight inside each column
// (arap_fit_kernel); the update of Eq. 22, W^k = (W_merge + lambda W_ARAP) / (1 + lambda),
// lambda = (1 + sigma^2) / (1 + 100); the cost of Eq. 21 summed over the nodes.  A device flag
// stops the iterations once the cost rises (the previous warps are kept); later launches of
// the loop then do nothing.
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

constexpr int kArapFitThreads = 256;   // a warp per node
constexpr int kArapMaxNodes = 1 << 22;

// The ARAP warp of node i (Sec. III-D as printed; one warp, lanes over the nodes j).
// w_j = exp(-alpha |x_i,0 - x_j,0|^2); the columns of C_0 and C_t are w_j d0_j and w_j dt_j with
// d0_j = x_j,0 - x_i,0, dt_j = x_j,t - x_i,t, so C_t C_0^T = sum w_j^2 dt_j d0_j^T.  In 2-D
// the det = +1 rotation U V^T of ARAP1 maximises tr(R^T C_t C_0^T) and has the direction
// (trace, antisymmetric part) = (sum w^2 dt.d0, sum w^2 d0 x dt), so only those two enter.
// ARAP2: s = sqrt(sum w^2 |dt|^2 / sum w^2 |d0|^2).  ARAP3: t = sum_j w_j (x_j,t / s -
// R x_j,0) / sum_j w_j, summed as x_i,t / s - R x_i,0 + (sum w dt / s - R sum w d0) / W so
// that every sum is of node-centred offsets.  Every sum is reduced by one fixed butterfly.
// A node whose columns are all zero (every other node's weight underflows) has no ARAP warp:
// it takes its current warp, which leaves Eq. 22 without an ARAP pull for it.
__global__ void __launch_bounds__(kArapFitThreads) arap_fit_kernel(
    const float2 *__restrict__ x0, const float2 *__restrict__ xt, const float *__restrict__ w_cur,
    int nn, float alpha, const ArapState *__restrict__ st, float *__restrict__ w_arap)
{
    const int i = blockIdx.x * (kArapFitThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= nn || st->done) return;
    const float2 xi = x0[i], yi = xt[i];
    // dot, cross, |d0|^2, |dt|^2 (each times w^2); W, sum w d0, sum w dt
    float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int j = lane; j < nn; j += 32) {
        const float2 a = x0[j], b = xt[j];
        const float d0x = a.x - xi.x, d0y = a.y - xi.y;
        const float dtx = b.x - yi.x, dty = b.y - yi.y;
        const float w = expf(-alpha * (d0x * d0x + d0y * d0y));
        const float w2 = w * w;
        acc[0] = fmaf(w2, dtx * d0x + dty * d0y, acc[0]);
        acc[1] = fmaf(w2, d0x * dty - d0y * dtx, acc[1]);
        acc[2] = fmaf(w2, d0x * d0x + d0y * d0y, acc[2]);
        acc[3] = fmaf(w2, dtx * dtx + dty * dty, acc[3]);
        acc[4] += w;
        acc[5] = fmaf(w, d0x, acc[5]);
        acc[6] = fmaf(w, d0y, acc[6]);
        acc[7] = fmaf(w, dtx, acc[7]);
        acc[8] = fmaf(w, dty, acc[8]);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if (lane != 0) return;
    // ARAP1: half angle of the direction (a, b) without cancellation
    const float a = acc[0], b = acc[1];
    const float rho = hypotf(a, b);
    float h0, h1;
    if (a >= 0.f) { h0 = rho + a; h1 = b; }
    else if (b >= 0.f) { h0 = b; h1 = rho - a; }
    else { h0 = -b; h1 = a - rho; }
    const float hn = hypotf(h0, h1);
    float c = 1.f, sn = 0.f;
    if (hn > 0.f) { c = h0 / hn; sn = h1 / hn; }
    const float sc = sqrtf(acc[3] / acc[2]);                          // ARAP2
    const float ct = c * c - sn * sn, stt = 2.f * c * sn;
    const float W = acc[4];
    const float mx = acc[7] / sc - (ct * acc[5] - stt * acc[6]);      // ARAP3
    const float my = acc[8] / sc - (stt * acc[5] + ct * acc[6]);
    const float tx = yi.x / sc - (ct * xi.x - stt * xi.y) + mx / W;
    const float ty = yi.y / sc - (stt * xi.x + ct * xi.y) + my / W;
    float *out = w_arap + 8 * (size_t)i;
    if (!(acc[2] > 0.f) || !isfinite(sc) || !isfinite(tx) || !isfinite(ty)) {
        const float *cur = w_cur + 8 * (size_t)i;
#pragma unroll
        for (int k = 0; k < 8; ++k) out[k] = cur[k];
        return;
    }
    // the quaternion from R and t: real part (c, sn), dual part 1/2 t^ r
    out[0] = c;
    out[1] = sn;
    out[2] = 0.5f * (tx * c + ty * sn);
    out[3] = 0.5f * (ty * c - tx * sn);
    out[4] = sc;
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
    size_t xt, warap, state, total;
};

ArapLayout arap_layout(int nn)
{
    auto al = [](size_t v) { return emdq_host::align_up(v, 256); };
    ArapLayout L;
    L.xt = 0;
    L.warap = L.xt + al(sizeof(float2) * (size_t)nn);
    L.state = L.warap + al(sizeof(float) * 8 * (size_t)nn);
    L.total = L.state + 256;
    return L;
}

}  // namespace emdq

using namespace emdq;
using namespace emdq_host;

extern "C" size_t emdq_arap_workspace_size(int nn)
{
    if (nn < 3 || nn > kArapMaxNodes) return 0;
    return arap_layout(nn).total;
}

extern "C" emdq_status emdq_arap_smooth(const float *x0, const float *w_merge, const float *s2,
                                        int nn, float alpha, int max_iters, float *w_out,
                                        void *workspace, size_t workspace_bytes, void *stream)
{
    if (!x0 || !w_merge || !s2 || !w_out || nn < 3 || max_iters < 0 || !(alpha > 0.f) ||
        !std::isfinite(alpha) || !aligned(x0, 8) || !aligned(w_out, 16))
        return EMDQ_EINVAL;
    if (nn > kArapMaxNodes) return EMDQ_ENOTSUP;
    const ArapLayout L = arap_layout(nn);
    if (!workspace || workspace_bytes < L.total || !aligned(workspace, 256)) return EMDQ_EWORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    auto *xt = reinterpret_cast<float2 *>(ws + L.xt);
    auto *wa = reinterpret_cast<float *>(ws + L.warap);
    auto *state = reinterpret_cast<ArapState *>(ws + L.state);
    if (cudaMemcpyAsync(w_out, w_merge, sizeof(float) * 8 * (size_t)nn, cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess)
        return EMDQ_ECUDA;
    arap_init_kernel<<<1, 1, 0, st>>>(state);
    const auto *x0f = reinterpret_cast<const float2 *>(x0);
    const int fit_blocks = (nn + kArapFitThreads / 32 - 1) / (kArapFitThreads / 32);
    for (int k = 0; k < max_iters; ++k) {
        arap_positions_kernel<<<(nn + 255) / 256, 256, 0, st>>>(x0f, w_out, nn, state, xt);
        arap_fit_kernel<<<fit_blocks, kArapFitThreads, 0, st>>>(x0f, xt, w_out, nn, alpha, state, wa);
        arap_update_kernel<<<1, kArapThreads, 0, st>>>(x0f, w_merge, s2, wa, nn, state, w_out);
    }
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}
