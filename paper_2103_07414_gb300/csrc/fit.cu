// EMDQ fit on the GPU: one cooperative, persistent launch runs step 0 and every EM
// iteration, synchronising its CTAs with bounded grid barriers, so that a whole fit costs
// one launch and no host round trip.
//
// Work split per iteration (N matches, G CTAs of 8 warps):
//   E-step      every CTA computes all N posteriors redundantly into shared memory
//               (identical inputs and reduction order, hence identical convergence
//               decisions in every CTA without an extra barrier)
//   M-step      warp w fits rows i = w, w + 8G, ..., two rows at a time so that each
//               shared-memory load of match j serves both.  The weighted similarity fit
//               needs the centred second moments of Eqs. 18-19; accumulating raw moments
//               and centring afterwards cancels catastrophically (it is why an FP64 finish
//               would be needed).  Instead the moments are taken about a shift close to
//               the weighted centroid -- at step 0 the centroid itself from a first pass,
//               later the previous round's centroid -- so nothing cancels and FP32
//               products and sums suffice.
//   barrier
//   residuals   warp w computes the leave-one-out blend at x_j for its rows j, four rows
//               at a time, blending the warp rows relative to row 0's (exact: the blend is
//               linear) to keep the FP32 sums small                  -> e_j (global)
//   barrier
//   sigma^2, gamma from the per-CTA partial sums, in a fixed order.
//
// Arithmetic per match pair: coordinates are staged pre-multiplied by
// k = sqrt(alpha log2 e) and the weights p as log2 p, so the Gaussian weight
// p_j exp(-alpha |x_i - x_j|^2) = 2^(log2 p_j - |k x_i - k x_j|^2) costs two FMAs and one
// MUFU.EX2; the (x, y) pairs of the moment sums use Blackwell's packed FP32x2 FMA/ADD/MUL
// (two lanes of arithmetic per instruction).
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace emdq {

// Block size: 256 threads when two CTAs fit an SM (the fit's shared memory is 44 bytes per
// match), 512 when only one does, so an SM keeps 16 warps either way.
constexpr int kFitThreadsSmall = 256;
constexpr int kFitThreadsLarge = 512;
constexpr int kFitMaxN = 5120;         // shared memory: 44 bytes per match
constexpr int kFitSmemPerMatch = 44;
constexpr int kFitMaxGrid = 1024;

struct FitArgs {
    const float2 *src;
    const float2 *dst;
    int n;
    float k;             // sqrt(alpha log2 e): staged coordinates are k x, k y
    float inv_k;
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
    float4 *cen;         // n weighted centroids of the last M-step, scaled local coordinates (workspace)
    float *partials;     // one float2 partial sum per CTA of the group (workspace)
    int *ord;            // n: the matches in Hilbert order; each CTA writes the positions of
                         // its own M-step rows (workspace)
    unsigned *bar;       // barrier arrival counter, zero at launch (workspace)
    int *flag;           // device status, zero at launch (workspace)
    unsigned spin_limit; // bound of every barrier wait (polls; kSpinLimit unless lowered)
    unsigned bar_extra;  // arrivals a barrier waits for beyond the grid's (0; 1 only to test
                         // the bounded wait: no barrier can then be passed)
};

struct FitSmem {
    float4 *q;           // warp rows minus row 0's: (r_w, r_z, d_x, d_y)
    float2 *x, *y;       // k x_j, k y_j
    float *p;            // posteriors
    float *lp;           // log2 of the posteriors (-inf for 0)
    float *qs;           // scale column of the warp rows minus row 0's
};

__device__ __forceinline__ FitSmem fit_smem(int n)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FitSmem s;
    s.q = reinterpret_cast<float4 *>(smem_raw);
    s.x = reinterpret_cast<float2 *>(s.q + n);
    s.y = s.x + n;
    s.p = reinterpret_cast<float *>(s.y + n);
    s.lp = s.p + n;
    s.qs = s.lp + n;
    return s;
}

// Grid-wide barrier with a bounded wait.  `epoch` counts barriers passed (same in every
// CTA).  Waits for ncta + extra arrivals per barrier, at most spin_limit polls.  Returns
// false if this CTA gave up waiting (the status flag is then ETIMEOUT).
__device__ bool grid_barrier(unsigned *bar, int *flag, unsigned &epoch, int ncta,
                             unsigned spin_limit, unsigned extra)
{
    __shared__ int timed_out;
    __syncthreads();
    epoch += 1;
    if (threadIdx.x == 0) {
        timed_out = 0;
        const unsigned target = epoch * (static_cast<unsigned>(ncta) + extra);
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        unsigned spins = 0;
        while (ld_acquire_gpu(bar) < target) {
            if (++spins > spin_limit) {
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

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Warp totals of K values of each of 4 rows (v[r][k]): two halving steps over the row index
// (across lanes 1 and 2 apart every lane keeps the rows of its own lane bits and sends the
// others), then butterflies over the remaining lane bits.  Lane L ends with the K totals of
// row L & 3, after 9K shuffles instead of the 20K of one butterfly per value; the order of
// the additions is fixed, so a row's totals are the same bits on every call.
template <int K>
__device__ __forceinline__ void rows4_sum(const float (&v)[4][K], int lane, float (&t)[K])
{
    const bool b0 = lane & 1, b1 = lane & 2;
    float h[2][K];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float keep = b0 ? v[2 * p + 1][k] : v[2 * p][k];
            const float send = b0 ? v[2 * p][k] : v[2 * p + 1][k];
            h[p][k] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float keep = b1 ? h[1][k] : h[0][k];
        const float send = b1 ? h[0][k] : h[1][k];
        t[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
    }
}

// Largest squared distance (scaled units) of a row from its group's origin for which the
// row's Gaussian weights are taken from the expanded exponent (mstep_group, residual_rows).
constexpr float kExpandMax = 4.f;

// Gaussian weight 2^(lp - |d|^2) of a scaled offset d.
__device__ __forceinline__ float gauss_w(float2 d, float lp)
{
    return ex2_ftz(fmaf(-d.x, d.x, fmaf(-d.y, d.y, lp)));
}

// Eqs. 18-20 for row i from the weight W, the weighted centroids relative to (x_i, y_i)
// in scaled coordinates, and the centred moments (scaled; the factor k^2 cancels in every
// ratio): rotation (2-D closed form of the SVD solution), scale (norm ratio), translation.
// The calling lane writes the q row and the centroid.
__device__ __forceinline__ void mstep_finish(const FitArgs &A, int i, float W, float ab0,
                                             float ab1, float bb0, float bb1, float vx, float vy,
                                             float dot, float cross)
{
    // Eq. 18 in 2-D: the rotation angle th maximising tr(R^T C_t C_0^T) has direction
    // (a, b) = (c00 + c11, c10 - c01); its half angle (the DQ real part) is the direction
    // of (rho + a, b), or of (b, rho - a) when a < 0 (no cancellation).
    const float a = dot, b = cross;
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
    // Eq. 20: t = ybar / s - R xbar, in pixels (the centroids unscaled onto the exact
    // match coordinates)
    const float2 xi = __ldg(A.src + i), yi = __ldg(A.dst + i);
    const float ct = c * c - sn * sn, st = 2.f * c * sn;
    const float xg0 = fmaf(ab0, A.inv_k, xi.x), xg1 = fmaf(ab1, A.inv_k, xi.y);
    const float yg0 = fmaf(bb0, A.inv_k, yi.x), yg1 = fmaf(bb1, A.inv_k, yi.y);
    const float tx = yg0 / sc - (ct * xg0 - st * xg1);
    const float ty = yg1 / sc - (st * xg0 + ct * xg1);
    const bool ok = W > 0.f && isfinite(W) && vx > 0.f && isfinite(sc) && isfinite(tx) &&
                    isfinite(ty);
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

// M-step of R rows that lie next to each other (consecutive in the Hilbert order of the
// matches; one warp, lanes over j): weights om_j = p_j exp(-alpha |x_j - x_i|^2).  The
// similarity fit needs the moments about each row's weighted centroid; summing raw moments
// and centring afterwards would cancel.  Here the moments of all R rows are summed about one
// origin o, the previous round's weighted centroid of the group's first row (at step 0 that
// centroid comes from a first pass), so the offsets u = x_j - o_x, v = y_j - o_y and the
// products |u|^2, |v|^2, u.v, u x v are formed once per j for the R rows.  Neighbouring rows
// have neighbouring centroids, so every row's centroid lies close to o compared with the
// spread of its weights, and moving its moments from o to that centroid afterwards cancels
// nothing.  Of C_t C_0^T only the trace (sum om u.v) and the antisymmetric part (sum om u x v)
// enter the 2-D rotation, so only those are summed.
// The totals of a row group as one lane keeps them until its row is finished: the nine sums
// about the group's origin, the origin (negated: x, y parts) and the row (-1: none).
struct RowSums {
    float t[9];
    float2 nox, noy;
    int i;
};

// Eqs. 18-20 for the row a lane holds (see mstep_group): the moments moved from the group's
// origin to the row's centroid, then the closed form.
__device__ __forceinline__ void mstep_row(const FitArgs &A, const FitSmem &S, const RowSums &k)
{
    if (k.i < 0) return;
    const float w = k.t[0], su0 = k.t[1], su1 = k.t[2], sv0 = k.t[3], sv1 = k.t[4];
    float vx = k.t[5], vy = k.t[6], dot = k.t[7], cross = k.t[8];
    // move the moments from o to the row's centroid o + d: m_c = m_o - W d d'^T
    float du0 = 0.f, du1 = 0.f, dv0 = 0.f, dv1 = 0.f;
    if (w > 0.f) {
        const float inv = 1.f / w;
        du0 = su0 * inv;
        du1 = su1 * inv;
        dv0 = sv0 * inv;
        dv1 = sv1 * inv;
    }
    vx -= w * (du0 * du0 + du1 * du1);
    vy -= w * (dv0 * dv0 + dv1 * dv1);
    dot -= w * (dv0 * du0 + dv1 * du1);
    cross -= w * (dv1 * du0 - dv0 * du1);
    // the centroid relative to (x_i, y_i): o + d - x_i
    const float2 xi = S.x[k.i], yi = S.y[k.i];
    mstep_finish(A, k.i, w, du0 - (k.nox.x + xi.x), du1 - (k.nox.y + xi.y),
                 dv0 - (k.noy.x + yi.x), dv1 - (k.noy.y + yi.y), vx, vy, dot, cross);
}

// The sums of a group of R rows (R <= 4); afterwards lane 4 slot + r keeps row r's totals in
// `keep` (the group's slot among the warp's groups waiting to be finished, slot < 8), so that
// the closed forms of up to 32 rows are then evaluated at once, one row per lane
// (mstep_row), instead of four lanes finishing four rows after every group.
template <int R>
__device__ void mstep_group(const FitArgs &A, const FitSmem &S, const int *rows, int lane,
                            bool first, int slot, RowSums &keep)
{
    const int n = A.n;
    float2 nxi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) nxi[r] = neg2(S.x[rows[r]]);
    const float2 x0 = S.x[rows[0]], y0 = S.y[rows[0]];
    float4 sh = first ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldcg(A.cen + rows[0]);
    if (first) {
        // the first row's weighted centroid, relative to (x_i0, y_i0)
        const float2 ny0 = neg2(y0);
        float W = 0.f;
        float2 sa = make_float2(0.f, 0.f), sb = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int j = lane; j < n; j += 32) {
            const float2 a = __fadd2_rn(S.x[j], nxi[0]);
            const float om = gauss_w(a, S.lp[j]);
            const float2 om2 = make_float2(om, om);
            W += om;
            sa = __ffma2_rn(om2, a, sa);
            sb = __ffma2_rn(om2, __fadd2_rn(S.y[j], ny0), sb);
        }
        const float w = warp_sum_f(W);
        const float a0 = warp_sum_f(sa.x), a1 = warp_sum_f(sa.y);
        const float b0 = warp_sum_f(sb.x), b1 = warp_sum_f(sb.y);
        if (w > 0.f && isfinite(w)) sh = make_float4(a0 / w, a1 / w, b0 / w, b1 / w);
    }
    // the origin o (negated, for adds), staged coordinates
    const float2 nox = make_float2(-(x0.x + sh.x), -(x0.y + sh.y));
    const float2 noy = make_float2(-(y0.x + sh.z), -(y0.y + sh.w));
    float W[R];
    float2 su[R], sv[R], sq[R], sc[R];     // sums of om u, om v, om (|u|^2, |v|^2), om (u.v, u x v)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        W[r] = 0.f;
        su[r] = sv[r] = sq[r] = sc[r] = make_float2(0.f, 0.f);
    }
    // The Gaussian exponent about o: with e = x_i - o and u = x_j - o,
    //     lp_j - |x_j - x_i|^2 = (lp_j - |u|^2) + 2 e.u - |e|^2,
    // where |u|^2 is one of the moment features and the last term is the same for every j of
    // row i: a factor 2^(-|e|^2) common to the row's nine sums, which every ratio of Eqs.
    // 18-20 cancels.  So the row's weights are taken as om 2^(|e|^2) = 2^((lp_j - |u|^2) +
    // 2 e.u): two FMAs per pair, where the offset x_j - x_i took a two-lane add more.  Used
    // when every row of the group lies within |e|^2 <= kExpandMax of o (scaled units; 2^4
    // at most as factor, and the rounding of the expanded exponent, about 2^-24 (|u|^2 +
    // 2 |e.u|), stays near 2^-20 for the pairs of non-negligible weight); other groups sum
    // the offsets as before.
    float2 e2[R];
    float emax = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float2 e = __fadd2_rn(neg2(nxi[r]), nox);
        emax = fmaxf(emax, fmaf(e.x, e.x, e.y * e.y));
        e2[r] = make_float2(2.f * e.x, 2.f * e.y);
    }
    if (emax <= kExpandMax) {
#pragma unroll 2
        for (int j = lane; j < n; j += 32) {
            const float2 xj = S.x[j], yj = S.y[j];
            const float lpj = S.lp[j];
            const float2 u = __fadd2_rn(xj, nox), v = __fadd2_rn(yj, noy);
            const float uu = fmaf(u.x, u.x, u.y * u.y);
            const float2 g1 = make_float2(uu, fmaf(v.x, v.x, v.y * v.y));
            const float2 g2 = make_float2(fmaf(u.x, v.x, u.y * v.y), fmaf(u.x, v.y, -(u.y * v.x)));
            const float cj = lpj - uu;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float om = ex2_ftz(fmaf(e2[r].x, u.x, fmaf(e2[r].y, u.y, cj)));
                const float2 om2 = make_float2(om, om);
                W[r] += om;
                su[r] = __ffma2_rn(om2, u, su[r]);
                sv[r] = __ffma2_rn(om2, v, sv[r]);
                sq[r] = __ffma2_rn(om2, g1, sq[r]);
                sc[r] = __ffma2_rn(om2, g2, sc[r]);
            }
        }
    } else {
#pragma unroll 2
        for (int j = lane; j < n; j += 32) {
            const float2 xj = S.x[j], yj = S.y[j];
            const float lpj = S.lp[j];
            const float2 u = __fadd2_rn(xj, nox), v = __fadd2_rn(yj, noy);
            const float2 g1 = make_float2(fmaf(u.x, u.x, u.y * u.y), fmaf(v.x, v.x, v.y * v.y));
            const float2 g2 = make_float2(fmaf(u.x, v.x, u.y * v.y), fmaf(u.x, v.y, -(u.y * v.x)));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float om = gauss_w(__fadd2_rn(xj, nxi[r]), lpj);
                const float2 om2 = make_float2(om, om);
                W[r] += om;
                su[r] = __ffma2_rn(om2, u, su[r]);
                sv[r] = __ffma2_rn(om2, v, sv[r]);
                sq[r] = __ffma2_rn(om2, g1, sq[r]);
                sc[r] = __ffma2_rn(om2, g2, sc[r]);
            }
        }
    }
    // the warp totals of the R rows: lanes 4 slot .. 4 slot + R - 1 keep them
    float v9[4][9], t[9];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const bool on = r < R;
        v9[r][0] = on ? W[r < R ? r : 0] : 0.f;
        v9[r][1] = on ? su[r < R ? r : 0].x : 0.f;
        v9[r][2] = on ? su[r < R ? r : 0].y : 0.f;
        v9[r][3] = on ? sv[r < R ? r : 0].x : 0.f;
        v9[r][4] = on ? sv[r < R ? r : 0].y : 0.f;
        v9[r][5] = on ? sq[r < R ? r : 0].x : 0.f;
        v9[r][6] = on ? sq[r < R ? r : 0].y : 0.f;
        v9[r][7] = on ? sc[r < R ? r : 0].x : 0.f;
        v9[r][8] = on ? sc[r < R ? r : 0].y : 0.f;
    }
    rows4_sum<9>(v9, lane, t);
    if ((lane >> 2) != slot) return;
    const int r = lane & 3;
    int i = -1;
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
        if (r == rr) i = rows[rr];
    keep.i = i;
#pragma unroll
    for (int k = 0; k < 9; ++k) keep.t[k] = t[k];
    keep.nox = nox;
    keep.noy = noy;
}

// Hilbert index of (x, y), 16 bits each (the curve of order 16: consecutive indices are
// neighbouring cells).  Quadrant by quadrant from the top bit, rotating and reflecting the
// remaining coordinates into the quadrant's frame.
__device__ __forceinline__ unsigned hilbert_index(unsigned x, unsigned y)
{
    unsigned d = 0;
    for (unsigned s = 1u << 15; s > 0; s >>= 1) {
        const unsigned rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        d += s * s * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = 0xffffu - x;
                y = 0xffffu - y;
            }
            const unsigned t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

// Leave-one-out residuals of R rows j (one warp, lanes over i; lane r < R accumulates
// row r's p e and p into pe, ps).  The blend at x_j of all
// rows i != j is taken relative to row 0 (S.q holds q_i - q_0), so the sums stay small.
// The loop sums over every i, the term i = j included, and that term -- computed bit for
// bit as in the loop -- is subtracted afterwards; where the rest of the weight is smaller
// than that term (an isolated match), the subtraction would cancel and the sum over
// i != j is taken again exactly.
// The rows of a group are neighbours in the Hilbert order; their Gaussian exponents are
// expanded about the first row's position o, as in the M-step: with e = x_j - o and
// u = x_i - o, lp_i - |x_i - x_j|^2 = (lp_i - |u|^2) + 2 e.u - |e|^2, and the factor
// 2^(-|e|^2), common to the row's six sums, cancels in the blend and in the comparison of
// the own term with the rest.  Groups whose rows lie farther than kExpandMax from o sum
// the offsets x_i - x_j as before.
// The totals of a residual row as one lane keeps them until the row is evaluated: the six
// sums over every i (the term i = j included), the group's origin (negated; NaN: offsets
// summed directly) and the row (-1: none).
struct ResSums {
    float t[6];
    float2 no;
    int j;
};

// Lane 4 slot + r keeps row r's totals in `keep` (slot < 8, the group's place among the
// warp's groups waiting), so that up to 32 residuals are then evaluated at once, one row per
// lane (residual_finish), instead of four lanes after every group.
template <int R>
__device__ void residual_rows(const FitArgs &A, const FitSmem &S, const int *rows, int lane,
                              int slot, ResSums &keep)
{
    const int n = A.n;
    float2 nxj[R], A1[R], A2[R];
    float W[R], As[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        nxj[r] = neg2(S.x[rows[r]]);
        A1[r] = A2[r] = make_float2(0.f, 0.f);
        W[r] = As[r] = 0.f;
    }
    const float2 no = nxj[0];
    float2 e2[R];
    float emax = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float2 e = __fadd2_rn(neg2(nxj[r]), no);
        emax = fmaxf(emax, fmaf(e.x, e.x, e.y * e.y));
        e2[r] = make_float2(2.f * e.x, 2.f * e.y);
    }
    // (a group of one row gains nothing: its origin is the row itself, e = 0)
    const bool expand = R >= 2 && emax <= kExpandMax;
    if (expand) {
#pragma unroll 2
        for (int i = lane; i < n; i += 32) {
            const float2 xi = S.x[i];
            const float lpi = S.lp[i];
            const float4 qi = S.q[i];
            const float qsi = S.qs[i];
            const float2 qab = make_float2(qi.x, qi.y), quv = make_float2(qi.z, qi.w);
            const float2 u = __fadd2_rn(xi, no);
            const float ci = fmaf(-u.x, u.x, fmaf(-u.y, u.y, lpi));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float w = ex2_ftz(fmaf(e2[r].x, u.x, fmaf(e2[r].y, u.y, ci)));
                const float2 w2 = make_float2(w, w);
                W[r] += w;
                A1[r] = __ffma2_rn(w2, qab, A1[r]);
                A2[r] = __ffma2_rn(w2, quv, A2[r]);
                As[r] = fmaf(w, qsi, As[r]);
            }
        }
    } else {
#pragma unroll 2
        for (int i = lane; i < n; i += 32) {
            const float2 xi = S.x[i];
            const float lpi = S.lp[i];
            const float4 qi = S.q[i];
            const float qsi = S.qs[i];
            const float2 qab = make_float2(qi.x, qi.y), quv = make_float2(qi.z, qi.w);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float w = gauss_w(__fadd2_rn(xi, nxj[r]), lpi);
                const float2 w2 = make_float2(w, w);
                W[r] += w;
                A1[r] = __ffma2_rn(w2, qab, A1[r]);
                A2[r] = __ffma2_rn(w2, quv, A2[r]);
                As[r] = fmaf(w, qsi, As[r]);
            }
        }
    }
    // the warp totals of the R rows: lanes 4 slot .. 4 slot + R - 1 keep them
    float v6[4][6], t[6];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const bool on = r < R;
        const int rr = r < R ? r : 0;
        v6[r][0] = on ? W[rr] : 0.f;
        v6[r][1] = on ? A1[rr].x : 0.f;
        v6[r][2] = on ? A1[rr].y : 0.f;
        v6[r][3] = on ? A2[rr].x : 0.f;
        v6[r][4] = on ? A2[rr].y : 0.f;
        v6[r][5] = on ? As[rr] : 0.f;
    }
    rows4_sum<6>(v6, lane, t);
    if ((lane >> 2) != slot) return;
    const int r = lane & 3;
    int j = -1;
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
        if (r == rr) j = rows[rr];
    keep.j = j;
    keep.no = expand ? no : make_float2(NAN, NAN);
#pragma unroll
    for (int k = 0; k < 6; ++k) keep.t[k] = t[k];
}

// The leave-one-out residual of the row each lane keeps (all lanes of the warp take part:
// isolated rows are summed again by the whole warp); adds p e and p of its row to pe, ps.
__device__ void residual_finish(const FitArgs &A, const FitSmem &S, const ResSums &keep, int lane,
                                float4 q0, float qs0, float &pe, float &ps)
{
    const int n = A.n;
    const bool has = keep.j >= 0;
    const int jl = has ? keep.j : 0;
    const float *t = keep.t;
    // the term i = j, the same bits as in the loop: offset (0, 0), so its weight is exactly
    // 2^lp_j, or with the exponent expanded about o, the loop's expression at u = e
    float wjj;
    if (isnan(keep.no.x)) {
        wjj = ex2_ftz(S.lp[jl]);
    } else {
        const float2 u = __fadd2_rn(S.x[jl], keep.no);
        const float cj = fmaf(-u.x, u.x, fmaf(-u.y, u.y, S.lp[jl]));
        wjj = ex2_ftz(fmaf(2.f * u.x, u.x, fmaf(2.f * u.y, u.y, cj)));
    }
    const float4 qj = S.q[jl];
    const float qsj = S.qs[jl];
    float wl = t[0] - wjj;
    float c0 = fmaf(-wjj, qj.x, t[1]), c1 = fmaf(-wjj, qj.y, t[2]);
    float c2 = fmaf(-wjj, qj.z, t[3]), c3 = fmaf(-wjj, qj.w, t[4]);
    float c4 = fmaf(-wjj, qsj, t[5]);
    // isolated matches (the rest of the weight below the own term): the sum over i != j
    // taken again exactly, one flagged row at a time by the whole warp
    unsigned slow = __ballot_sync(0xffffffffu, has && !(wl >= wjj));
    while (slow) {
        const int r = __ffs(slow) - 1;
        slow &= slow - 1;
        const int j = __shfl_sync(0xffffffffu, jl, r);
        const float2 nx = neg2(S.x[j]);
        float w_ = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f, d4 = 0.f;
        for (int i = lane; i < n; i += 32) {
            if (i == j) continue;
            const float wi = gauss_w(__fadd2_rn(S.x[i], nx), S.lp[i]);
            const float4 qi = S.q[i];
            w_ += wi;
            d0 = fmaf(wi, qi.x, d0);
            d1 = fmaf(wi, qi.y, d1);
            d2 = fmaf(wi, qi.z, d2);
            d3 = fmaf(wi, qi.w, d3);
            d4 = fmaf(wi, S.qs[i], d4);
        }
        w_ = warp_sum_f(w_);
        d0 = warp_sum_f(d0);
        d1 = warp_sum_f(d1);
        d2 = warp_sum_f(d2);
        d3 = warp_sum_f(d3);
        d4 = warp_sum_f(d4);
        if (lane == r) {
            wl = w_; c0 = d0; c1 = d1; c2 = d2; c3 = d3; c4 = d4;
        }
    }
    if (!has) return;
    float e = INFINITY;
    if (wl > 0.f) {
        const float inv = 1.f / wl;
        const float2 xj = __ldg(A.src + jl), yj = __ldg(A.dst + jl);
        const float2 yh = apply_blend(fmaf(c0, inv, q0.x), fmaf(c1, inv, q0.y),
                                      fmaf(c2, inv, q0.z), fmaf(c3, inv, q0.w),
                                      fmaf(c4, inv, qs0), xj.x, xj.y);
        const float r0 = yj.x - yh.x, r1 = yj.y - yh.y;
        e = r0 * r0 + r1 * r1;
    }
    __stcg(A.e + jl, e);
    if (isfinite(e)) {
        pe += S.p[jl] * e;
        ps += S.p[jl];
    }
}

// Block-wide sums of two floats in a fixed order: warp butterflies, then every thread
// adds the NT/32 warp totals in warp order, so every thread (and every CTA, given the same
// inputs) holds the same bits.
template <int NT>
__device__ float2 block_sum2(float a, float b, float2 *red)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    a = warp_sum_f(a);
    b = warp_sum_f(b);
    if (lane == 0) red[w] = make_float2(a, b);
    __syncthreads();
    float2 t = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) {
        t.x += red[k].x;
        t.y += red[k].y;
    }
    __syncthreads();
    return t;
}

// Grid barrier, then the device status word as every thread of every CTA sees it.
__device__ int barrier_status(const FitArgs &A, unsigned &epoch, int *s_flag, int ncta)
{
    const bool ok = grid_barrier(A.bar, A.flag, epoch, ncta, A.spin_limit, A.bar_extra);
    if (threadIdx.x == 0) *s_flag = ok ? __ldcg(A.flag) : (int)EMDQ_ETIMEOUT;
    __syncthreads();
    return *s_flag;
}

// log2 of a posterior for the staged weights (-inf for 0: its weight 2^-inf is 0)
__device__ __forceinline__ float log2_p(float p) { return __log2f(p); }

// One fit on a group of `ncta` co-resident CTAs of NT threads; `rank` is this CTA's index
// in the group.
template <int NT>
// p0: the initial weights (null: all 1); max_iters: EM rounds this launch may run; iters_base:
// rounds run by earlier launches of the same fit (added to the reported count).  resume: the
// fit continues a launch that ran iters_base rounds without converging: p0 is its posterior,
// and its row order, centroids, residuals and its sigma^2 and gamma (the fit record) are the
// state after its last round, so step 0 is not run again and EM goes on with the next E-step.
__device__ __forceinline__ void fit_body(const FitArgs &A, int rank, int ncta, const float *p0,
                                         int max_iters, int iters_base, bool resume)
{
    constexpr int kWarps = NT / 32;
    const int n = A.n;
    const FitSmem S = fit_smem(n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gwarp = rank * kWarps + warp, nwarps = ncta * kWarps;
    __shared__ float2 red[kWarps];
    __shared__ int s_flag;
    unsigned epoch = 0;

    // stage the matches (scaled) and the initial weights; every CTA checks every input
    int bad = 0;
    float p0sum = 0.f;
    for (int j = threadIdx.x; j < n; j += NT) {
        const float2 x = A.src[j], y = A.dst[j];
        S.x[j] = make_float2(A.k * x.x, A.k * x.y);
        S.y[j] = make_float2(A.k * y.x, A.k * y.y);
        const float p = p0 ? p0[j] : 1.f;
        S.p[j] = p;
        S.lp[j] = p0 ? log2_p(p) : 0.f;
        p0sum += p;
        bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(y.x) && isfinite(y.y) && isfinite(p) &&
                 p >= 0.f);
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
    if (resume) gamma = __ldcg(&A.info->gamma);
    else if (p0) gamma = fminf(fmaxf(block_sum2<NT>(p0sum, 0.f, red).x / n, 0.05f), 0.95f);

    // The M-step rows of this CTA: positions [pb, pe) of the Hilbert order of the matches.
    // Every CTA sorts all the matches (the same order in each; the q staging area is free
    // until the first residual pass) and keeps the positions of its own rows.
    const int pb = static_cast<int>((long long)rank * n / ncta);
    const int pe = static_cast<int>((long long)(rank + 1) * n / ncta);
    if (resume) {
        // the order of the earlier launch (all n positions, written by its CTAs) stands
    } else if ((n + ncta - 1) / ncta <= kWarps) {
        // at most one row per warp in every CTA of the problem (the same decision in all of
        // them): every row is its own group (its origin its own previous centroid), so the
        // order of the rows changes nothing and the sort is skipped
        for (int t = pb + threadIdx.x; t < pe; t += NT) A.ord[t] = t;
        __syncthreads();
    } else {
        float2 lo = make_float2(INFINITY, INFINITY), hi = make_float2(-INFINITY, -INFINITY);
        for (int j = threadIdx.x; j < n; j += NT) {
            const float2 x = S.x[j];
            lo = make_float2(fminf(lo.x, x.x), fminf(lo.y, x.y));
            hi = make_float2(fmaxf(hi.x, x.x), fmaxf(hi.y, x.y));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
            lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
            hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
            hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
        }
        if (lane == 0) red[warp] = lo;
        __syncthreads();
        float2 blo = red[0];
        for (int k = 1; k < kWarps; ++k) blo = make_float2(fminf(blo.x, red[k].x), fminf(blo.y, red[k].y));
        __syncthreads();
        if (lane == 0) red[warp] = hi;
        __syncthreads();
        float2 bhi = red[0];
        for (int k = 1; k < kWarps; ++k) bhi = make_float2(fmaxf(bhi.x, red[k].x), fmaxf(bhi.y, red[k].y));
        __syncthreads();
        const float ext = fmaxf(bhi.x - blo.x, bhi.y - blo.y);
        const float qs = ext > 0.f ? 65535.f / ext : 0.f;
        unsigned long long *key = reinterpret_cast<unsigned long long *>(S.q);
        int P = 1;
        while (P < n) P <<= 1;                    // P <= 2n keys fit the 16 n bytes of S.q
        for (int t = threadIdx.x; t < P; t += NT) {
            unsigned long long k = ~0ull;
            if (t < n) {
                const float2 x = S.x[t];
                const unsigned hx = static_cast<unsigned>(fminf(fmaxf((x.x - blo.x) * qs, 0.f), 65535.f));
                const unsigned hy = static_cast<unsigned>(fminf(fmaxf((x.y - blo.y) * qs, 0.f), 65535.f));
                k = (static_cast<unsigned long long>(hilbert_index(hx, hy)) << 32) | static_cast<unsigned>(t);
            }
            key[t] = k;
        }
        __syncthreads();
        // bitonic sort of the P keys, ascending (keys are distinct: the index is the low word)
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = threadIdx.x; t < P / 2; t += NT) {
                    const int a = 2 * j * (t / j) + (t & (j - 1)), b = a + j;
                    const unsigned long long ka = key[a], kb = key[b];
                    if ((ka > kb) == ((a & k) == 0)) {
                        key[a] = kb;
                        key[b] = ka;
                    }
                }
                __syncthreads();
            }
        }
        for (int t = pb + threadIdx.x; t < pe; t += NT) A.ord[t] = static_cast<int>(key[t] & 0xffffffffu);
        __syncthreads();
    }
    // each warp takes groups of 4 consecutive positions (the same number per warp), then
    // one contiguous run of the remaining positions (at most 4)
    // (the closed forms of a warp's rows are evaluated 32 at a time, one row per lane, after
    // every 8 groups and at the end)
    auto mstep_all = [&](bool first) {
        const int m = pe - pb, per = m / (4 * kWarps);
        RowSums keep;
        keep.i = -1;
        int slot = 0;
        for (int g = 0; g < per; ++g) {
            const int b = pb + 4 * (warp + kWarps * g);
            const int rows[4] = {A.ord[b], A.ord[b + 1], A.ord[b + 2], A.ord[b + 3]};
            mstep_group<4>(A, S, rows, lane, first, slot, keep);
            if (++slot == 8) {
                mstep_row(A, S, keep);
                keep.i = -1;
                slot = 0;
            }
        }
        const int base = pb + 4 * kWarps * per, left = m - 4 * kWarps * per;
        const int lb = base + warp * left / kWarps, le = base + (warp + 1) * left / kWarps;
        if (le - lb == 4) {
            const int rows[4] = {A.ord[lb], A.ord[lb + 1], A.ord[lb + 2], A.ord[lb + 3]};
            mstep_group<4>(A, S, rows, lane, first, slot, keep);
        } else if (le - lb == 3) {
            const int rows[3] = {A.ord[lb], A.ord[lb + 1], A.ord[lb + 2]};
            mstep_group<3>(A, S, rows, lane, first, slot, keep);
        } else if (le - lb == 2) {
            const int rows[2] = {A.ord[lb], A.ord[lb + 1]};
            mstep_group<2>(A, S, rows, lane, first, slot, keep);
        } else if (le - lb == 1) {
            const int rows[1] = {A.ord[lb]};
            mstep_group<1>(A, S, rows, lane, first, slot, keep);
        }
        mstep_row(A, S, keep);
    };
    // residuals of this CTA's rows and its partial sums, then the barrier
    auto residuals_and_barrier = [&]() -> int {
        const float4 q0 = __ldcg(reinterpret_cast<const float4 *>(A.q_out));
        const float qs0 = __ldcg(A.q_out + 4);
        for (int i = threadIdx.x; i < n; i += NT) {
            const float4 r0 = __ldcg(reinterpret_cast<const float4 *>(A.q_out + 8 * (size_t)i));
            const float r4 = __ldcg(A.q_out + 8 * (size_t)i + 4);
            S.q[i] = make_float4(r0.x - q0.x, r0.y - q0.y, r0.z - q0.z, r0.w - q0.w);
            S.qs[i] = r4 - qs0;
        }
        __syncthreads();
        float pe = 0.f, ps = 0.f;
        ResSums keep;
        keep.j = -1;
        int slot = 0;
        // groups of R consecutive positions of the Hilbert order (every CTA's M-step positions
        // are written before the barrier that precedes this pass), dealt to the warps of the
        // whole group of CTAs in turn, R = 4 unless there are fewer than 4 rows per warp (then
        // as many as the warps have on average, at least one: every warp gets work); the last
        // group holds the positions left
        const int R = min(4, max(1, n / nwarps));
        for (int t = R * gwarp; t < n; t += R * nwarps) {
            const int left = min(R, n - t);
            if (left >= 4) {
                const int rows[4] = {__ldcg(A.ord + t), __ldcg(A.ord + t + 1), __ldcg(A.ord + t + 2),
                                     __ldcg(A.ord + t + 3)};
                residual_rows<4>(A, S, rows, lane, slot, keep);
            } else if (left == 3) {
                const int rows[3] = {__ldcg(A.ord + t), __ldcg(A.ord + t + 1), __ldcg(A.ord + t + 2)};
                residual_rows<3>(A, S, rows, lane, slot, keep);
            } else if (left == 2) {
                const int rows[2] = {__ldcg(A.ord + t), __ldcg(A.ord + t + 1)};
                residual_rows<2>(A, S, rows, lane, slot, keep);
            } else {
                const int rows[1] = {__ldcg(A.ord + t)};
                residual_rows<1>(A, S, rows, lane, slot, keep);
            }
            if (++slot == 8) {
                residual_finish(A, S, keep, lane, q0, qs0, pe, ps);
                keep.j = -1;
                slot = 0;
            }
        }
        residual_finish(A, S, keep, lane, q0, qs0, pe, ps);
        const float2 t = block_sum2<NT>(pe, ps, red);
        if (threadIdx.x == 0) __stcg(reinterpret_cast<float2 *>(A.partials) + rank, t);
        return barrier_status(A, epoch, &s_flag, ncta);
    };
    // after that barrier: sigma^2 from the per-CTA partials; every warp reduces the
    // partials itself, in the same order
    auto load_e_and_sigma2 = [&]() -> float {
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

    // step 0 (a resumed fit has its residuals and sigma^2 from the earlier launch)
    float sigma2 = A.sigma2_floor;
    int st = EMDQ_OK;
    if (resume) {
        sigma2 = __ldcg(&A.info->sigma2);
    } else {
        mstep_all(true);
        st = barrier_status(A, epoch, &s_flag, ncta);
        if (st < EMDQ_EDEGENERATE) st = residuals_and_barrier();
        if (st < EMDQ_EDEGENERATE) sigma2 = load_e_and_sigma2();
    }

    int it = 0;
    bool converged = false;
    const float two_pi = 6.28318530717958647692f;
    while (st < EMDQ_EDEGENERATE && it < max_iters) {
        ++it;
        // E-step: every CTA, all N posteriors
        float dpmax = 0.f, psum = 0.f;
        const float norm = 1.f / (two_pi * sigma2);
        const float outl = (1.f - gamma) * A.inv_area;
        for (int j = threadIdx.x; j < n; j += NT) {
            {
                const float e = __ldcg(A.e + j);      // all N residuals, from every CTA
                const float G = isfinite(e) ? expf(-e / (2.f * sigma2)) * norm : 0.f;
                const float pn = gamma * G / (gamma * G + outl);
                dpmax = fmaxf(dpmax, fabsf(pn - S.p[j]));
                S.p[j] = pn;
                S.lp[j] = log2_p(pn);
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
        for (int k = 0; k < kWarps; ++k) {
            dpall = fmaxf(dpall, red[k].x);
            ptot += red[k].y;
        }
        __syncthreads();
        const float gamma_next = fminf(fmaxf(ptot / n, 0.05f), 0.95f);
        // M-step with the new weights, then residuals and sigma^2
        mstep_all(false);
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
        for (int j = threadIdx.x; j < n; j += NT) {
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
            A.info->iters = iters_base + it;
            A.info->sigma2 = sigma2;
            A.info->gamma = gamma;
        }
    }
}

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) emdq_fit_kernel(FitArgs A)
{
    fit_body<NT>(A, blockIdx.x, gridDim.x, A.p0, A.max_iters, 0, false);
}

// Many fits in one cooperative launch: problem b runs on CTAs [b * group, (b + 1) * group),
// with its own barrier counter, status word and partial sums.
// Problem b owns CTAs [first[b], first[b + 1]): a split of the co-resident CTAs in
// proportion to each problem's work, so problems of different sizes finish together.
constexpr int kFitBatchMax = 64;
constexpr int kFitMaxPhases = 16;     // phases of emdq_fit_batch_phases
struct FitBatch {
    FitArgs a[kFitBatchMax];
    int first[kFitBatchMax + 1];
    int count;
};

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) emdq_fit_batch_kernel(const __grid_constant__ FitBatch B)
{
    int lo = 0, hi = B.count - 1;          // the problem whose CTA range holds blockIdx.x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.first[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const FitArgs &A = B.a[lo];
    fit_body<NT>(A, blockIdx.x - B.first[lo], B.first[lo + 1] - B.first[lo], A.p0, A.max_iters, 0, false);
}

// CTAs of NT threads a problem of n matches can use: one warp per row.
__host__ __device__ constexpr int fit_useful_ctas(int n, int nt) { return (n + nt / 32 - 1) / (nt / 32); }

// A later phase of a phased batch: the problems that ran `before` EM rounds without converging
// (status EMDQ_ENOCONV, before rounds) take every CTA of this launch, split in proportion to n^2
// (at least one each, at most one warp per row, largest remainders first), and each continues
// for at most `add` more rounds from the state its last round left: the posteriors p_out, the
// row order, centroids and residuals in the workspace, sigma^2 and gamma in its fit record.  It
// goes on with the next E-step, as one launch running every round would; only the split of the
// rows over CTAs (the M-step's groups, the order of the sigma^2 partial sums), and with it the
// FP32 rounding, differs.  Every CTA computes the same split; CTAs left over return at once.
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) emdq_fit_batch_next_kernel(const __grid_constant__ FitBatch B,
                                                                         int before, int add)
{
    __shared__ int pick[3];                 // this CTA's problem, rank and CTA count
    if (threadIdx.x == 0) {
        int ctas[kFitBatchMax];
        double rem[kFitBatchMax], wsum = 0.0;
        bool on[kFitBatchMax];
        for (int b = 0; b < B.count; ++b) {
            const emdq_fit_info *f = B.a[b].info;
            on[b] = __ldcg(&f->status) == EMDQ_ENOCONV && __ldcg(&f->iters) == before;
            if (on[b]) wsum += (double)B.a[b].n * (double)B.a[b].n;
        }
        const int total = gridDim.x;
        int used = 0;
        for (int b = 0; b < B.count; ++b) {
            ctas[b] = 0;
            rem[b] = -1.0;
            if (!on[b]) continue;
            const double share = total * ((double)B.a[b].n * (double)B.a[b].n) / wsum;
            const int cap = fit_useful_ctas(B.a[b].n, NT);
            int k = (int)share;
            if (k < 1) k = 1;
            if (k > cap) k = cap;
            ctas[b] = k;
            rem[b] = k < cap ? share - (double)k : -1.0;
            used += k;
        }
        while (used < total) {
            int best = -1;
            for (int b = 0; b < B.count; ++b)
                if (rem[b] >= 0.0 && ctas[b] < fit_useful_ctas(B.a[b].n, NT) && (best < 0 || rem[b] > rem[best]))
                    best = b;
            if (best < 0) break;
            ++ctas[best];
            rem[best] -= 1.0;
            ++used;
        }
        pick[0] = -1;
        for (int b = 0, first = 0; b < B.count; first += ctas[b], ++b)
            if (first <= (int)blockIdx.x && (int)blockIdx.x < first + ctas[b]) {
                pick[0] = b;
                pick[1] = blockIdx.x - first;
                pick[2] = ctas[b];
            }
    }
    __syncthreads();
    const int b = pick[0];
    if (b < 0) return;                      // no problem left for this CTA
    const FitArgs &A = B.a[b];
    fit_body<NT>(A, pick[1], pick[2], A.p_out, add, before, true);
}

}  // namespace emdq

using namespace emdq;
using namespace emdq_host;

namespace {
// Fit workspace: residuals e[n], centroids cen[n], per-CTA partial sums, the row order
// ord[n], then 256 bytes for the barrier counter and the status word.
struct FitLayout {
    size_t e_off, cen_off, part_off, ord_off, bar_off, total;
};
constexpr size_t al256(size_t v) { return (v + 255) / 256 * 256; }
constexpr FitLayout fit_layout(int n)
{
    const size_t e = al256(sizeof(float) * (size_t)n), cen = al256(sizeof(float4) * (size_t)n),
                 part = al256(sizeof(double) * 2 * kFitMaxGrid), ord = al256(sizeof(int) * (size_t)n);
    return FitLayout{0, e, e + cen, e + cen + part, e + cen + part + ord, e + cen + part + ord + 256};
}
size_t fit_smem_bytes(int n) { return (size_t)n * kFitSmemPerMatch; }

// The shared-memory limit of every fit kernel instance, raised once per device.
bool fit_attributes()
{
    static std::mutex mu;
    static int done_dev = -1;
    const DeviceInfo &D = device_info();
    if (D.device < 0) return false;
    std::lock_guard<std::mutex> g(mu);
    if (done_dev == D.device) return true;
    const int smax = (int)fit_smem_bytes(kFitMaxN);
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (cudaFuncSetAttribute(emdq_fit_kernel<kFitThreadsSmall>, attr, smax) != cudaSuccess ||
        cudaFuncSetAttribute(emdq_fit_kernel<kFitThreadsLarge>, attr, smax) != cudaSuccess ||
        cudaFuncSetAttribute(emdq_fit_batch_kernel<kFitThreadsSmall>, attr, smax) != cudaSuccess ||
        cudaFuncSetAttribute(emdq_fit_batch_kernel<kFitThreadsLarge>, attr, smax) != cudaSuccess ||
        cudaFuncSetAttribute(emdq_fit_batch_next_kernel<kFitThreadsSmall>, attr, smax) != cudaSuccess ||
        cudaFuncSetAttribute(emdq_fit_batch_next_kernel<kFitThreadsLarge>, attr, smax) != cudaSuccess)
        return false;
    done_dev = D.device;
    return true;
}

// Block size for `smem` bytes of shared memory per CTA (256 threads if two CTAs fit an SM,
// else 512) and the CTAs then co-resident on the device; false on error.
bool fit_shape(bool batch, size_t smem, int &nt, int &capacity)
{
    if (!fit_attributes()) return false;
    const DeviceInfo &D = device_info();
    int per = 0;
    const cudaError_t e =
        batch ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per, emdq_fit_batch_kernel<kFitThreadsSmall>, kFitThreadsSmall, smem)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per, emdq_fit_kernel<kFitThreadsSmall>, kFitThreadsSmall, smem);
    if (e != cudaSuccess) return false;
    if (per >= 2) {
        nt = kFitThreadsSmall;
        capacity = per * D.sms;
        return true;
    }
    const cudaError_t e2 =
        batch ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per, emdq_fit_batch_kernel<kFitThreadsLarge>, kFitThreadsLarge, smem)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per, emdq_fit_kernel<kFitThreadsLarge>, kFitThreadsLarge, smem);
    if (e2 != cudaSuccess || per < 1) return false;
    nt = kFitThreadsLarge;
    capacity = per * D.sms;
    return true;
}

// CTAs of nt threads a problem of n matches can use: one warp per row.
int useful_ctas(int n, int nt) { return fit_useful_ctas(n, nt); }
}  // namespace

extern "C" int emdq_fit_max_n(void) { return kFitMaxN; }

extern "C" size_t emdq_fit_workspace_size(int n)
{
    if (n < 0) return 0;
    return fit_layout(n).total;
}

namespace {
// The wait settings of emdq_params.reserved: [0] > 0 lowers the bound of every barrier wait to
// that many polls; [1] != 0 makes every barrier wait for one arrival more than the grid makes,
// so that no wait can end (a test of the bounded wait: the fit then reports ETIMEOUT).
void wait_hooks(const emdq_params &P, FitArgs &A)
{
    A.spin_limit = P.reserved[0] > 0 && static_cast<unsigned>(P.reserved[0]) < kSpinLimit
                       ? static_cast<unsigned>(P.reserved[0])
                       : kSpinLimit;
    A.bar_extra = P.reserved[1] != 0 ? 1u : 0u;
}
}  // namespace

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

    int nt = 0, cap = 0;
    if (!fit_shape(false, smem, nt, cap)) return EMDQ_ECUDA;
    int grid = useful_ctas(n, nt);
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
    A.k = static_cast<float>(std::sqrt(alpha * 1.4426950408889634074));
    A.inv_k = 1.f / A.k;
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
    A.ord = reinterpret_cast<int *>(ws + L.ord_off);
    A.bar = reinterpret_cast<unsigned *>(ws + L.bar_off);
    A.flag = reinterpret_cast<int *>(ws + L.bar_off + 64);
    wait_hooks(P, A);

    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = nt == kFitThreadsSmall
                              ? cudaLaunchKernelEx(&cfg, emdq_fit_kernel<kFitThreadsSmall>, A)
                              : cudaLaunchKernelEx(&cfg, emdq_fit_kernel<kFitThreadsLarge>, A);
    if (e != cudaSuccess) return EMDQ_ECUDA;
    return EMDQ_OK;
}


// ------------------------------------------------------------------ emdq_fit_batch -----
namespace {
// Batch workspace: one 256-byte header per problem (barrier counter, status word) packed
// first so that a single memset clears them all, then each problem's residuals and
// partial sums.
size_t batch_body_bytes(int n)
{
    return fit_layout(n).bar_off;      // e, cen, partials, ord; the headers are packed first
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

namespace {


// Split `total` CTAs of nt threads over the problems in proportion to n^e (e = expo), at
// least one each and at most useful_ctas(n, nt); largest remainders take the leftovers.
void split_ctas(const emdq_fit_problem *problems, int count, int total, int nt, double expo,
                int *ctas)
{
    double wsum = 0.0;
    for (int b = 0; b < count; ++b) wsum += std::pow((double)problems[b].n, expo);
    double rem[kFitBatchMax];
    int used = 0;
    for (int b = 0; b < count; ++b) {
        const double share = total * std::pow((double)problems[b].n, expo) / wsum;
        int k = (int)share;
        const int cap = useful_ctas(problems[b].n, nt);
        if (k < 1) k = 1;
        if (k > cap) k = cap;
        ctas[b] = k;
        rem[b] = k < cap ? share - (double)k : -1.0;
        used += k;
    }
    while (used < total) {
        int best = -1;
        for (int b = 0; b < count; ++b)
            if (rem[b] >= 0.0 && ctas[b] < useful_ctas(problems[b].n, nt) &&
                (best < 0 || rem[b] > rem[best]))
                best = b;
        if (best < 0) break;
        ++ctas[best];
        rem[best] -= 1.0;
        ++used;
    }
    while (used > total) {                 // at least one CTA each overshot the capacity
        int best = -1;
        for (int b = 0; b < count; ++b)
            if (ctas[b] > 1 && (best < 0 || ctas[b] > ctas[best])) best = b;
        if (best < 0) break;
        --ctas[best];
        --used;
    }
}

}  // namespace

namespace {

// The checks, the CTA split and the per-problem arguments of a batched fit; on success B, nt
// (threads per CTA), smem and cap (co-resident CTAs) are set and every problem's barrier words
// are cleared on st.
emdq_status fit_batch_setup(const emdq_fit_problem *problems, int count, const emdq_params &P,
                            const int *ctas, void *workspace, size_t workspace_bytes,
                            cudaStream_t st, FitBatch &B, int &nt, size_t &smem, int &cap)
{
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
    smem = fit_smem_bytes(max_n);
    if (smem > D.smem_optin) return EMDQ_ENOTSUP;
    nt = 0;
    cap = 0;
    if (!fit_shape(true, smem, nt, cap)) return EMDQ_ECUDA;
    if (count > cap) return EMDQ_ENOTSUP;     // more problems than co-resident CTAs

    B.count = count;
    {
        int split[kFitBatchMax];
        if (ctas) {
            int sum = 0;
            for (int b = 0; b < count; ++b) {
                if (ctas[b] < 1 || ctas[b] > kFitMaxGrid) return EMDQ_EINVAL;
                sum += ctas[b];
            }
            if (sum > cap) return EMDQ_EINVAL;     // would not be co-resident
            for (int b = 0; b < count; ++b) split[b] = ctas[b];
        } else {
            split_ctas(problems, count, cap, nt, 2.0, split);   // EM work grows as n^2
        }
        B.first[0] = 0;
        for (int b = 0; b < count; ++b) B.first[b + 1] = B.first[b] + split[b];
    }

    char *ws = static_cast<char *>(workspace);
    if (cudaMemsetAsync(ws, 0, 256 * (size_t)count, st) != cudaSuccess) return EMDQ_ECUDA;
    size_t off = 256 * (size_t)count;
    const double log2e = 1.4426950408889634074;
    for (int b = 0; b < count; ++b) {
        const emdq_fit_problem &q = problems[b];
        FitArgs &A = B.a[b];
        A.src = reinterpret_cast<const float2 *>(q.src);
        A.dst = reinterpret_cast<const float2 *>(q.dst);
        A.n = q.n;
        const double alpha = P.alpha > 0.f ? P.alpha : emdq_alpha_for_frame(q.frame_w, q.frame_h);
        A.k = static_cast<float>(std::sqrt(alpha * log2e));
        A.inv_k = 1.f / A.k;
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
        wait_hooks(P, A);
        const FitLayout L = fit_layout(q.n);
        A.e = reinterpret_cast<float *>(ws + off + L.e_off);
        A.cen = reinterpret_cast<float4 *>(ws + off + L.cen_off);
        A.partials = reinterpret_cast<float *>(ws + off + L.part_off);
        A.ord = reinterpret_cast<int *>(ws + off + L.ord_off);
        off += batch_body_bytes(q.n);
    }
    return EMDQ_OK;
}

// One cooperative launch of `grid` CTAs: the first phase (add < 0: every problem from its p0,
// its own CTA range) or a later one (the problems unconverged after `before` rounds, `add`
// more rounds).
emdq_status fit_batch_launch(const FitBatch &B, int grid, int nt, size_t smem, cudaStream_t st,
                             int before, int add)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (add < 0)
        e = nt == kFitThreadsSmall ? cudaLaunchKernelEx(&cfg, emdq_fit_batch_kernel<kFitThreadsSmall>, B)
                                   : cudaLaunchKernelEx(&cfg, emdq_fit_batch_kernel<kFitThreadsLarge>, B);
    else
        e = nt == kFitThreadsSmall
                ? cudaLaunchKernelEx(&cfg, emdq_fit_batch_next_kernel<kFitThreadsSmall>, B, before, add)
                : cudaLaunchKernelEx(&cfg, emdq_fit_batch_next_kernel<kFitThreadsLarge>, B, before, add);
    return e == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

}  // namespace

extern "C" emdq_status emdq_fit_batch_ex(const emdq_fit_problem *problems, int count,
                                         const emdq_params *prm, const int *ctas, void *workspace,
                                         size_t workspace_bytes, void *stream)
{
    emdq_params P;
    emdq_default_params(&P);
    if (prm) P = *prm;
    static thread_local FitBatch B;
    int nt = 0, cap = 0;
    size_t smem = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const emdq_status rc = fit_batch_setup(problems, count, P, ctas, workspace, workspace_bytes, st,
                                           B, nt, smem, cap);
    if (rc != EMDQ_OK) return rc;
    return fit_batch_launch(B, B.first[count], nt, smem, st, 0, -1);
}

extern "C" emdq_status emdq_fit_batch_phases(const emdq_fit_problem *problems, int count,
                                             const emdq_params *prm, const int *phase_iters,
                                             int nphases, void *workspace, size_t workspace_bytes,
                                             void *stream)
{
    if (!phase_iters || nphases < 1 || nphases > kFitMaxPhases) return EMDQ_EINVAL;
    for (int k = 0; k < nphases; ++k)
        if (phase_iters[k] < 1 || (k > 0 && phase_iters[k] <= phase_iters[k - 1])) return EMDQ_EINVAL;
    if (problems && count >= 1 && count <= kFitBatchMax)
        for (int b = 0; b < count; ++b)
            if (!problems[b].p_out) return EMDQ_EINVAL;     // the next phase starts from it
    emdq_params P;
    emdq_default_params(&P);
    if (prm) P = *prm;
    P.max_iters = phase_iters[0];
    static thread_local FitBatch B;
    int nt = 0, cap = 0;
    size_t smem = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    emdq_status rc = fit_batch_setup(problems, count, P, nullptr, workspace, workspace_bytes, st, B,
                                     nt, smem, cap);
    if (rc != EMDQ_OK) return rc;
    rc = fit_batch_launch(B, B.first[count], nt, smem, st, 0, -1);
    if (rc != EMDQ_OK || nphases == 1) return rc;
    // later phases: every co-resident CTA of the continuation kernel
    int per = 0;
    const cudaError_t e = nt == kFitThreadsSmall
                              ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &per, emdq_fit_batch_next_kernel<kFitThreadsSmall>, nt, smem)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &per, emdq_fit_batch_next_kernel<kFitThreadsLarge>, nt, smem);
    if (e != cudaSuccess || per < 1) return EMDQ_ECUDA;
    int grid = per * device_info().sms;
    if (grid > cap) grid = cap;
    for (int k = 1; k < nphases; ++k) {
        // the barrier words start every launch at zero
        if (cudaMemsetAsync(workspace, 0, 256 * (size_t)count, st) != cudaSuccess) return EMDQ_ECUDA;
        rc = fit_batch_launch(B, grid, nt, smem, st, phase_iters[k - 1],
                              phase_iters[k] - phase_iters[k - 1]);
        if (rc != EMDQ_OK) return rc;
    }
    return EMDQ_OK;
}

extern "C" emdq_status emdq_fit_batch(const emdq_fit_problem *problems, int count,
                                      const emdq_params *prm, void *workspace,
                                      size_t workspace_bytes, void *stream)
{
    return emdq_fit_batch_ex(problems, count, prm, nullptr, workspace, workspace_bytes, stream);
}

extern "C" int emdq_fit_batch_capacity(const emdq_fit_problem *problems, int count)
{
    if (!problems || count < 1 || count > kFitBatchMax) return 0;
    int max_n = 0;
    for (int b = 0; b < count; ++b) max_n = problems[b].n > max_n ? problems[b].n : max_n;
    if (max_n < 1 || max_n > kFitMaxN) return 0;
    int nt = 0, cap = 0;
    return fit_shape(true, fit_smem_bytes(max_n), nt, cap) ? cap : 0;
}

extern "C" emdq_status emdq_fit_batch_autotune(const emdq_fit_problem *problems, int count,
                                               const emdq_params *prm, void *workspace,
                                               size_t workspace_bytes, void *stream, int reps,
                                               int *ctas_out, float *ms_out)
{
    if (!ctas_out || reps < 1 || reps > 100) return EMDQ_EINVAL;
    if (!problems || count < 1 || count > kFitBatchMax) return EMDQ_EINVAL;
    int max_n = 0;
    for (int b = 0; b < count; ++b) max_n = problems[b].n > max_n ? problems[b].n : max_n;
    if (max_n < 3 || max_n > kFitMaxN) return EMDQ_ENOTSUP;
    int nt = 0, cap = 0;
    if (!fit_shape(true, fit_smem_bytes(max_n), nt, cap)) return EMDQ_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return EMDQ_EINVAL;                    // times launches: not inside a capture
    // candidates: CTAs in proportion to n^e, and all CTAs or the useful ones only
    const double expos[] = {0.0, 1.0, 1.5, 2.0, 2.5, 3.0};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return EMDQ_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return EMDQ_ECUDA;
    }
    float best = -1.f;
    emdq_status rc = EMDQ_OK;
    int split[kFitBatchMax];
    for (double expo : expos) {
        split_ctas(problems, count, cap, nt, expo, split);
        // one untimed launch, then the best of `reps`
        rc = emdq_fit_batch_ex(problems, count, prm, split, workspace, workspace_bytes, stream);
        if (rc != EMDQ_OK) break;
        float t_best = -1.f;
        for (int r = 0; r < reps && rc == EMDQ_OK; ++r) {
            if (cudaEventRecord(e0, st) != cudaSuccess) { rc = EMDQ_ECUDA; break; }
            rc = emdq_fit_batch_ex(problems, count, prm, split, workspace, workspace_bytes, stream);
            if (rc != EMDQ_OK) break;
            float ms = 0.f;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = EMDQ_ECUDA;
                break;
            }
            if (t_best < 0.f || ms < t_best) t_best = ms;
        }
        if (rc != EMDQ_OK) break;
        if (best < 0.f || t_best < best) {
            best = t_best;
            for (int b = 0; b < count; ++b) ctas_out[b] = split[b];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == EMDQ_OK && ms_out) *ms_out = best;
    return rc;
}

// ------------------------------------------------------------------ emdq_fit_noalloc ---
// The same fit for callers that must not allocate device memory: its scratch (residuals,
// per-CTA partial sums, barrier counter, status word) lives in one fixed array in this
// library's device memory, sized for the largest fit (kFitMaxN matches), instead of a
// caller workspace.  Every GPU that loads the library holds the array until exit.
namespace {

constexpr size_t kNoAllocScratchBytes = fit_layout(kFitMaxN).total;   // about 136 KB

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
    // the argument errors of emdq_fit come first, so that a bad argument gives EMDQ_EINVAL
    // whatever n is; only then is a valid n checked against the array (fit_layout grows with
    // n, so n <= kFitMaxN bounds the scratch a fit needs)
    emdq_params P;
    emdq_default_params(&P);
    if (prm) P = *prm;
    if (!src || !dst || !q_out || !c_out || !info || n < 3 || frame_w < 1 || frame_h < 1 ||
        P.max_iters < 0 || !(P.tol_p >= 0.f) || !(P.sigma2_floor > 0.f))
        return EMDQ_EINVAL;
    if (!aligned(src, 8) || !aligned(dst, 8) || !aligned(q_out, 16) || !aligned(info, 4))
        return EMDQ_EINVAL;
    if (n > kFitMaxN) return EMDQ_ENOTSUP;   // beyond the fixed scratch array
    void *ws = noalloc_scratch();
    if (!ws) return EMDQ_ECUDA;
    // emdq_fit clears the barrier counter and status word before its launch
    return emdq_fit(src, dst, n, frame_w, frame_h, prm, p0, q_out, c_out, p_out, info, ws,
                    kNoAllocScratchBytes, stream);
}
