// Deformation-node tracking and merging (Sec. III-A/C, App. A, Eqs. 5, 8, 9, 12-15).
//
// emdq_node_track: one warp per node.  The node's position at t-1, p = W_i,t-1(x_i,0); the
// lanes sum the Eqs. 2-3 blend of the t-1 -> t EMDQ warps at p (FP32 weights c_j
// exp(-alpha |p - x_j|^2)) and the nearest inlier's squared distance (Eq. 8); lane 0 composes
// W_i,t = f(W_i,t-1, dW) -- scale ds s_old, rotation by the product of the two half-angle unit
// complex numbers, translation dR t_old + dt / s_old (App. A's requirement s_new q_new(x) =
// ds dq(s_old q_old(x))) -- and propagates sigma^2 = ds^2 sigma_old^2 + exp(beta d^2) (Eq. 9).
// emdq_node_merge: one thread per node, the EKF merge of Eqs. 12-15 in closed form for the
// 2 x 2 covariance.
// emdq_node_restrict: one warp per node, the bound of Eq. 11 by every feature.
// emdq_feature_uncertainty: one warp per feature, Eq. 10 (the leave-one-out field of the other
// inliers at the feature: an inlier's squared error, or an outlier's scale and Eq. 8).
// emdq_keyframe_distances: one block per key frame, Eq. 6's mean node distance.
// emdq_hex_nodes (host) and emdq_node_init: the node insertion of Sec. III-E -- the hexagonal
// lattice grown breadth-first from the image centre over the 6 neighbours of every node, and a
// new node's warp as the ARAP-weighted average of the existing nodes' (one warp per new node).
#include <cmath>
#include <deque>
#include <set>
#include <utility>

#include "common.cuh"

namespace emdq {

// planar DQ row (r_w, r_z, d_x, d_y) with a unit real part: translation t = 2 (d_x c - d_y s,
// d_x s + d_y c) for r = (c, s)
struct Sim {
    float c, s;      // half-angle unit complex number (r_w, r_z)
    float tx, ty;    // translation (inside the scale)
    float sc;        // scale
};

__device__ __forceinline__ Sim sim_from_row(float rw, float rz, float dx, float dy, float sc)
{
    const float nr = rsqrtf(rw * rw + rz * rz);
    Sim m;
    m.c = rw * nr;
    m.s = rz * nr;
    const float ux = dx * nr, uy = dy * nr;
    m.tx = 2.f * (ux * m.c - uy * m.s);
    m.ty = 2.f * (ux * m.s + uy * m.c);
    m.sc = sc;
    return m;
}

__device__ __forceinline__ void row_from_sim(const Sim &m, float *row)
{
    float c = m.c, s = m.s;
    if (c < 0.f) {
        c = -c;
        s = -s;
    }
    row[0] = c;
    row[1] = s;
    row[2] = 0.5f * (m.tx * c + m.ty * s);
    row[3] = 0.5f * (-m.tx * s + m.ty * c);
    row[4] = m.sc;
    row[5] = 1.f;
    row[6] = 0.f;
    row[7] = 0.f;
}

// x -> s (R x + t); R from the half-angle number (cos th = c^2 - s^2, sin th = 2 c s)
__device__ __forceinline__ float2 sim_apply(const Sim &m, float x, float y)
{
    const float ct = m.c * m.c - m.s * m.s, st = 2.f * m.c * m.s;
    return make_float2(m.sc * (ct * x - st * y + m.tx), m.sc * (st * x + ct * y + m.ty));
}

constexpr int kNodeWarps = 8;

__global__ void __launch_bounds__(32 * kNodeWarps) node_track_kernel(
    const float2 *__restrict__ x0, const float *__restrict__ w_old, const float *__restrict__ s2_old,
    int nn, const float *__restrict__ q, const float *__restrict__ c, const float2 *__restrict__ src,
    int n, float alpha, float beta, float *__restrict__ w_new, float *__restrict__ s2_new)
{
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kNodeWarps + (threadIdx.x >> 5);
    if (i >= nn) return;
    const float *wo = w_old + 8 * (size_t)i;
    const Sim mo = sim_from_row(wo[0], wo[1], wo[2], wo[3], wo[4]);
    const float2 x = x0[i];
    const float2 p = sim_apply(mo, x.x, x.y);
    float sw = 0.f, ss = 0.f, s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, dmin = INFINITY;
    for (int j = lane; j < n; j += 32) {
        const float cj = c[j];
        const float2 xj = src[j];
        const float dx = xj.x - p.x, dy = xj.y - p.y, d2 = dx * dx + dy * dy;
        const float w = cj * expf(-alpha * d2);
        const float4 qj = *reinterpret_cast<const float4 *>(q + 8 * (size_t)j);
        const float sj = q[8 * (size_t)j + 4];
        sw += w;
        ss = fmaf(w, sj, ss);
        s0 = fmaf(w, qj.x, s0);
        s1 = fmaf(w, qj.y, s1);
        s2 = fmaf(w, qj.z, s2);
        s3 = fmaf(w, qj.w, s3);
        if (cj > 0.f) dmin = fminf(dmin, d2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
        dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
    }
    if (lane != 0) return;
    float *wn = w_new + 8 * (size_t)i;
    if (!(sw > 0.f) || !isfinite(sw)) {
        for (int k = 0; k < 8; ++k) wn[k] = wo[k];
        s2_new[i] = INFINITY;
        return;
    }
    const Sim md = sim_from_row(s0, s1, s2, s3, ss / sw);
    // App. A: rotation dth + th_old (half-angle numbers multiply), translation dR t_old + dt / s_old
    Sim mn;
    mn.c = md.c * mo.c - md.s * mo.s;
    mn.s = md.c * mo.s + md.s * mo.c;
    const float ct = md.c * md.c - md.s * md.s, st = 2.f * md.c * md.s;
    mn.tx = ct * mo.tx - st * mo.ty + md.tx / mo.sc;
    mn.ty = st * mo.tx + ct * mo.ty + md.ty / mo.sc;
    mn.sc = md.sc * mo.sc;
    row_from_sim(mn, wn);
    s2_new[i] = md.sc * md.sc * s2_old[i] + expf(beta * dmin);
}

__global__ void node_merge_kernel(const float2 *__restrict__ x0, const float *__restrict__ w_track,
                                  const float *__restrict__ s2_track,
                                  const float *__restrict__ w_loop,
                                  const float *__restrict__ s2_loop, const float *__restrict__ w_key,
                                  int nn, float gamma, float *__restrict__ w_out,
                                  float *__restrict__ s2_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const float *wt = w_track + 8 * (size_t)i, *wl = w_loop + 8 * (size_t)i,
                *wk = w_key + 8 * (size_t)i;
    const float2 x = x0[i];
    const Sim mt = sim_from_row(wt[0], wt[1], wt[2], wt[3], wt[4]);
    const Sim mk = sim_from_row(wk[0], wk[1], wk[2], wk[3], wk[4]);
    const float2 xt = sim_apply(mt, x.x, x.y), xk = sim_apply(mk, x.x, x.y);
    const float ddx = xt.x - xk.x, ddy = xt.y - xk.y;
    const float eta = expf(-gamma * (ddx * ddx + ddy * ddy));      // Eq. 13
    const float vt = s2_track[i], vl = s2_loop[i];
    const float a01 = eta * sqrtf(vt) * sqrtf(vl);                  // Eq. 12
    // A^-1 [1 1]^T = (vl - a01, vt - a01) / det; sum(A^-1) = (vt + vl - 2 a01) / det
    const float den = vt + vl - 2.f * a01;
    const float w0 = (vl - a01) / den, w1 = (vt - a01) / den;         // Eq. 15
    const float det = vt * vl - a01 * a01;
    const float sm = det / den;                                        // Eq. 14
    float *wo = w_out + 8 * (size_t)i;
    if (!(w0 >= 0.f) || !(w1 >= 0.f) || !isfinite(sm) || !(det > 0.f)) {
        const bool t = vt <= vl;
        const float *pick = t ? wt : wl;
        for (int k = 0; k < 8; ++k) wo[k] = pick[k];
        s2_out[i] = t ? vt : vl;
        return;
    }
    const float nt = rsqrtf(wt[0] * wt[0] + wt[1] * wt[1]), nl = rsqrtf(wl[0] * wl[0] + wl[1] * wl[1]);
    float qv[4];
    for (int k = 0; k < 4; ++k) qv[k] = w0 * wt[k] * nt + w1 * wl[k] * nl;
    const float nq = rsqrtf(qv[0] * qv[0] + qv[1] * qv[1]);
    for (int k = 0; k < 4; ++k) wo[k] = qv[k] * nq;
    wo[4] = w0 * wt[4] + w1 * wl[4];
    wo[5] = 1.f;
    wo[6] = 0.f;
    wo[7] = 0.f;
    s2_out[i] = sm;
}

__global__ void __launch_bounds__(32 * kNodeWarps) node_restrict_kernel(
    const float2 *__restrict__ x, const float *__restrict__ s2, int nn, const float2 *__restrict__ y,
    const float *__restrict__ s2f, int m, float beta, float *__restrict__ s2_out)
{
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kNodeWarps + (threadIdx.x >> 5);
    if (i >= nn) return;
    const float2 xi = x[i];
    float best = INFINITY;
    for (int j = lane; j < m; j += 32) {
        const float2 yj = y[j];
        const float dx = xi.x - yj.x, dy = xi.y - yj.y;
        best = fminf(best, s2f[j] + expf(beta * (dx * dx + dy * dy)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) s2_out[i] = fminf(s2[i], best);
}

__global__ void __launch_bounds__(32 * kNodeWarps) feature_uncertainty_kernel(
    const float2 *__restrict__ src, const float2 *__restrict__ dst, int n,
    const float *__restrict__ q, const float *__restrict__ c, float alpha, float beta,
    const float *__restrict__ s2_prev, float *__restrict__ s2_out)
{
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * kNodeWarps + (threadIdx.x >> 5);
    if (j >= n) return;
    const float2 xj = src[j];
    float sw = 0.f, ss = 0.f, s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, dmin = INFINITY;
    for (int i = lane; i < n; i += 32) {
        if (i == j) continue;                  // leave one out (an outlier weighs 0 anyway)
        const float ci = c[i];
        const float2 xi = src[i];
        const float dx = xi.x - xj.x, dy = xi.y - xj.y, d2 = dx * dx + dy * dy;
        const float w = ci * expf(-alpha * d2);
        const float4 qi = *reinterpret_cast<const float4 *>(q + 8 * (size_t)i);
        sw += w;
        ss = fmaf(w, q[8 * (size_t)i + 4], ss);
        s0 = fmaf(w, qi.x, s0);
        s1 = fmaf(w, qi.y, s1);
        s2 = fmaf(w, qi.z, s2);
        s3 = fmaf(w, qi.w, s3);
        if (ci > 0.f) dmin = fminf(dmin, d2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
        dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
    }
    if (lane != 0) return;
    if (!(sw > 0.f) || !isfinite(sw)) {
        s2_out[j] = INFINITY;
        return;
    }
    const Sim m = sim_from_row(s0, s1, s2, s3, ss / sw);
    if (c[j] > 0.f) {
        const float2 yh = sim_apply(m, xj.x, xj.y);
        const float2 yj = dst[j];
        const float ex = yj.x - yh.x, ey = yj.y - yh.y;
        s2_out[j] = s2_prev[j] + (ex * ex + ey * ey);
    } else {
        s2_out[j] = m.sc * m.sc * s2_prev[j] + expf(beta * dmin);
    }
}

__global__ void __launch_bounds__(32 * kNodeWarps) node_init_kernel(
    const float2 *__restrict__ x0, const float *__restrict__ w, int nn, const float2 *__restrict__ pts,
    int np, float alpha, float *__restrict__ w_out)
{
    const int lane = threadIdx.x & 31;
    const int k = blockIdx.x * kNodeWarps + (threadIdx.x >> 5);
    if (k >= np) return;
    const float2 p = pts[k];
    float sw = 0.f, ss = 0.f, s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int j = lane; j < nn; j += 32) {
        const float2 xj = x0[j];
        const float dx = xj.x - p.x, dy = xj.y - p.y;
        const float g = expf(-alpha * (dx * dx + dy * dy));
        const float *wj = w + 8 * (size_t)j;
        sw += g;                             // Eqs. 2-3 with every weight 1
        ss = fmaf(g, wj[4], ss);
        s0 = fmaf(g, wj[0], s0);
        s1 = fmaf(g, wj[1], s1);
        s2 = fmaf(g, wj[2], s2);
        s3 = fmaf(g, wj[3], s3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    }
    if (lane != 0) return;
    float *o = w_out + 8 * (size_t)k;
    if (!(sw > 0.f) || !isfinite(sw)) {
        for (int m = 0; m < 8; ++m) o[m] = __int_as_float(0x7fffffff);
        return;
    }
    const float nq = rsqrtf(s0 * s0 + s1 * s1);
    o[0] = s0 * nq;
    o[1] = s1 * nq;
    o[2] = s2 * nq;
    o[3] = s3 * nq;
    o[4] = ss / sw;
    o[5] = 1.f;
    o[6] = 0.f;
    o[7] = 0.f;
}

constexpr int kKeyThreads = 256;

__global__ void __launch_bounds__(kKeyThreads) keyframe_distances_kernel(
    const float2 *__restrict__ xt, const float2 *__restrict__ xk, int nn, float *__restrict__ out)
{
    __shared__ float red[kKeyThreads / 32];
    const float2 *k = xk + (size_t)blockIdx.x * nn;
    float sum = 0.f;
    for (int i = threadIdx.x; i < nn; i += kKeyThreads) sum += hypotf(xt[i].x - k[i].x, xt[i].y - k[i].y);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < kKeyThreads / 32; ++w) t += red[w];
        out[blockIdx.x] = t / static_cast<float>(nn);
    }
}

}  // namespace emdq

using namespace emdq;
using namespace emdq_host;

extern "C" float emdq_gamma_for_frame(int w, int h)
{
    // Sec. III-G: gamma = 5e-3 / s^2 (Eq. 13), the resolution scale of alpha and beta
    const double s = (w / 480.0 + h / 270.0) / 2.0;
    return static_cast<float>(5e-3 / (s * s));
}

extern "C" emdq_status emdq_node_track(const float *x0, const float *w_old, const float *s2_old,
                                       int nn, const float *q, const float *c, const float *src,
                                       int n, float alpha, float beta, float *w_new,
                                       float *s2_new, void *stream)
{
    if (nn < 0 || n < 0 || !(alpha > 0.f) || !(beta > 0.f) || !std::isfinite(alpha) ||
        !std::isfinite(beta))
        return EMDQ_EINVAL;
    if (nn == 0) return EMDQ_OK;
    if (!x0 || !w_old || !s2_old || !w_new || !s2_new || !aligned(x0, 8) ||
        (n > 0 && (!q || !c || !src || !aligned(q, 16) || !aligned(src, 8))))
        return EMDQ_EINVAL;
    node_track_kernel<<<(nn + kNodeWarps - 1) / kNodeWarps, 32 * kNodeWarps, 0,
                        static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float2 *>(x0), w_old, s2_old, nn, q, c,
        reinterpret_cast<const float2 *>(src), n, alpha, beta, w_new, s2_new);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

extern "C" emdq_status emdq_node_merge(const float *x0, const float *w_track,
                                       const float *s2_track, const float *w_loop,
                                       const float *s2_loop, const float *w_key, int nn,
                                       float gamma, float *w_out, float *s2_out, void *stream)
{
    if (nn < 0 || !(gamma > 0.f) || !std::isfinite(gamma)) return EMDQ_EINVAL;
    if (nn == 0) return EMDQ_OK;
    if (!x0 || !w_track || !s2_track || !w_loop || !s2_loop || !w_key || !w_out || !s2_out ||
        !aligned(x0, 8))
        return EMDQ_EINVAL;
    node_merge_kernel<<<(nn + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float2 *>(x0), w_track, s2_track, w_loop, s2_loop, w_key, nn, gamma,
        w_out, s2_out);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

extern "C" emdq_status emdq_node_restrict(const float *x, const float *s2, int nn, const float *y,
                                          const float *s2f, int m, float beta, float *s2_out,
                                          void *stream)
{
    if (nn < 0 || m < 0 || !(beta > 0.f) || !std::isfinite(beta)) return EMDQ_EINVAL;
    if (nn == 0) return EMDQ_OK;
    if (!x || !s2 || !s2_out || !aligned(x, 8) || (m > 0 && (!y || !s2f || !aligned(y, 8))))
        return EMDQ_EINVAL;
    node_restrict_kernel<<<(nn + kNodeWarps - 1) / kNodeWarps, 32 * kNodeWarps, 0,
                           static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float2 *>(x), s2, nn, reinterpret_cast<const float2 *>(y), s2f, m,
        beta, s2_out);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

extern "C" emdq_status emdq_keyframe_distances(const float *xt, const float *xk, int nn, int nk,
                                               float *out, void *stream)
{
    if (nn < 1 || nk < 0 || !xt || !aligned(xt, 8) || (nk > 0 && (!xk || !out || !aligned(xk, 8))))
        return EMDQ_EINVAL;
    if (nk == 0) return EMDQ_OK;
    keyframe_distances_kernel<<<nk, kKeyThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float2 *>(xt), reinterpret_cast<const float2 *>(xk), nn, out);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

extern "C" emdq_status emdq_feature_uncertainty(const float *src, const float *dst, int n,
                                                const float *q, const float *c, float alpha,
                                                float beta, const float *s2_prev, float *s2_out,
                                                void *stream)
{
    if (n < 0 || !(alpha > 0.f) || !(beta > 0.f) || !std::isfinite(alpha) || !std::isfinite(beta))
        return EMDQ_EINVAL;
    if (n == 0) return EMDQ_OK;
    if (!src || !dst || !q || !c || !s2_prev || !s2_out || !aligned(src, 8) || !aligned(dst, 8) ||
        !aligned(q, 16))
        return EMDQ_EINVAL;
    feature_uncertainty_kernel<<<(n + kNodeWarps - 1) / kNodeWarps, 32 * kNodeWarps, 0,
                                 static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float2 *>(src), reinterpret_cast<const float2 *>(dst), n, q, c, alpha,
        beta, s2_prev, s2_out);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

extern "C" int emdq_hex_nodes(int w, int h, float spacing, float *x0_out, int capacity)
{
    if (w < 1 || h < 1 || !(spacing > 0.f) || !std::isfinite(spacing) || capacity < 0 ||
        (capacity > 0 && !x0_out))
        return -1;
    // lattice row r at y = cy + r dy, odd rows shifted by s/2; kept: points within the covering
    // radius s/sqrt(3) of the frame [0, w-1] x [0, h-1]
    const double s = spacing, dy = s * std::sqrt(3.0) / 2.0, m = s / std::sqrt(3.0);
    const double cx = (w - 1) / 2.0, cy = (h - 1) / 2.0;
    auto pos = [&](int r, int k, double &x, double &y) {
        y = cy + r * dy;
        x = cx + ((r & 1) ? 0.5 * s : 0.0) + k * s;
    };
    auto keep = [&](int r, int k) {
        double x, y;
        pos(r, k, x, y);
        const double ex = std::max(std::max(-x, 0.0), x - (w - 1));
        const double ey = std::max(std::max(-y, 0.0), y - (h - 1));
        return ex * ex + ey * ey <= m * m;
    };
    std::set<std::pair<int, int>> seen;
    std::deque<std::pair<int, int>> todo;
    seen.insert({0, 0});
    todo.push_back({0, 0});
    int count = 0;
    while (!todo.empty()) {
        const auto [r, k] = todo.front();
        todo.pop_front();
        if (count < capacity) {
            double x, y;
            pos(r, k, x, y);
            x0_out[2 * count] = static_cast<float>(x);
            x0_out[2 * count + 1] = static_cast<float>(y);
        }
        ++count;
        if (count > (1 << 26)) return -1;           // spacing far too small for the frame
        // the 6 neighbours in the odd-row-shifted layout
        const int k0 = (r & 1) ? k : k - 1, k1 = k0 + 1;
        const std::pair<int, int> nb[6] = {{r, k - 1}, {r, k + 1}, {r - 1, k0}, {r - 1, k1},
                                           {r + 1, k0}, {r + 1, k1}};
        for (const auto &q : nb)
            if (!seen.count(q) && keep(q.first, q.second)) {
                seen.insert(q);
                todo.push_back(q);
            }
    }
    return count;
}

extern "C" emdq_status emdq_node_init(const float *x0, const float *w, int nn, const float *pts,
                                      int npts, float alpha, float *w_out, void *stream)
{
    if (nn < 1 || npts < 0 || !(alpha > 0.f) || !std::isfinite(alpha)) return EMDQ_EINVAL;
    if (npts == 0) return EMDQ_OK;
    if (!x0 || !w || !pts || !w_out || !aligned(x0, 8) || !aligned(pts, 8)) return EMDQ_EINVAL;
    node_init_kernel<<<(npts + kNodeWarps - 1) / kNodeWarps, 32 * kNodeWarps, 0,
                       static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float2 *>(x0), w, nn, reinterpret_cast<const float2 *>(pts), npts,
        alpha, w_out);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}
