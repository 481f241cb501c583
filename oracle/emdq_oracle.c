/*
 * FP64 CPU oracle of the EMDQ field + mosaic path.  TEST INFRASTRUCTURE ONLY (see
 * emdq_oracle.h): loaded by the tests, the smoke check and the benchmark's CPU-baseline
 * leg, never by the product library.  It shares no code with the CUDA path.
 *
 * What it follows
 *   Eq. 1 (and its footnote)  warp = scale x planar dual quaternion, x' = s (R x + t)
 *   Eqs. 2-4                  pixel warp = Gaussian-weighted linear blend of the match warps
 *   Eqs. 16-20                weighted closed-form similarity fit (rotation from the SVD of
 *                             C_t C_0^T, scale as the norm ratio, translation as the weighted
 *                             average of X_t / s - R X_0), then "the quaternion from R and t"
 *   Sec. III-F, Eqs. 23-24    frame 0 inserted directly; per-pixel gather and a running
 *                             average whose weight is capped at 30
 *   Sec. III-G                alpha = 2e-4 / s^2, beta = 3e-3 / s^2, s = (w/480 + h/270)/2
 *   Sec. III-C, Eq. 8         uncertainty of the EMDQ field at a point: the minimum over the
 *                             feature inliers of exp(beta d^2), d the distance to the inlier
 *   Eq. 5, App. A, Eq. 9      node tracking: W_i,t = f(W_i,t-1, dW_i) with f the composition
 *                             s_new q_new(x) = ds dq(s_old q_old(x)); sigma^2 propagation
 *   Eqs. 12-15                EKF merge of the tracking and loop-closing node warps
 *   Eq. 10                    feature uncertainty: an inlier adds its squared EMDQ error, an
 *                             outlier propagates as a node does (Eq. 9)
 *   Eq. 11                    node uncertainty bounded by the features': sigma_i^2 <=
 *                             sigma_j,feature^2 + exp(beta d_ij^2) for every feature j
 *   Eq. 6                     key-frame distance: mean over the nodes of |x_i,t - x_i,k|
 *   Sec. III-E                new nodes: a hexagonal lattice grown from the image centre; a new
 *                             node's warp is the ARAP-weighted average of the existing nodes'
 *   Sec. III-D, Eqs. 16-22    ARAP smoothing of the node warps; the ARAP warp of a node is
 *                             Eqs. 16-17 and ARAP1-3 as printed: columns w_j^i (x_j - x_i)
 *                             centred on node i, the weight inside each column
 *
 * Readings (the paper is silent, garbled or delegates to its EMDQ reference)
 *   - Eq. 3 blends q without normalising it; a blended DQ is normalised by the norm of its
 *     real part before use (dual-quaternion blending).  In the planar case the real and
 *     dual parts are orthogonal, so that is the whole normalisation.
 *   - Eqs. 16-17 put the weight inside each column of C_0, C_t, centred on node i.  The EM
 *     M-step (EMDQ's own fit, which the paper does not print) centres on the weighted
 *     centroids and applies each weight once (weighted least squares); the ARAP fit of
 *     Sec. III-D keeps the printed columns.  In both the rotation is the det=+1 solution,
 *     written in 2-D closed form.
 *   - The EM iteration itself (the paper treats EMDQ as a black box):
 *       step 0   p_j = 1 (or a given p0); M-step; leave-one-out residuals e_j;
 *                sigma^2 = max(sum p e / (2 sum p), floor); gamma = 0.5
 *       repeat   posterior p_j = gamma G_j / (gamma G_j + (1 - gamma)/(w h)),
 *                  G_j = exp(-e_j / (2 sigma^2)) / (2 pi sigma^2)       (E-step)
 *                M-step with weights p_j exp(-alpha |x_i - x_j|^2)       (M-step)
 *                leave-one-out residuals, sigma^2 update, gamma = clamp(mean p, .05, .95)
 *                stop when max |dp| < tol or after max_iters iterations
 *       output   c_i = p_i if p_i >= 0.5 else 0 (the inliers the field interpolates among)
 *     Residuals that have no leave-one-out support (weight sum 0) are +inf: they get
 *     posterior 0 and are left out of the sigma^2 sums.
 *   - Eq. 23 lacks its normalisation and Eq. 24 prints max{w+1, 30}: the blend is the
 *     running average c <- round((w c + v)/(w + 1)), w <- min(w + 1, 30); an empty pixel
 *     takes round(v).  round(z) = floor(z + 0.5), clamped to [0, 255].
 *   - The warp is a gather: canvas pixel p (reference coordinates) samples frame t at
 *     u = p + d(p), which equals the paper's inverse map wherever W_p is invertible.  A
 *     sample is valid iff 0 <= u_x <= w-1 and 0 <= u_y <= h-1; taps beyond the last
 *     row/column are clamped (their weight is 0).  Invalid samples leave the canvas pixel
 *     untouched.
 */
#include "emdq_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

double orc_alpha_for_frame(int w, int h)
{
    double s = (w / 480.0 + h / 270.0) / 2.0;
    return 2e-4 / (s * s);
}

double orc_beta_for_frame(int w, int h)
{
    double s = (w / 480.0 + h / 270.0) / 2.0;
    return 3e-3 / (s * s);
}

/* Hamilton product of quaternions stored (w, x, y, z). */
static void qmul(const double a[4], const double b[4], double o[4])
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

void orc_dq_from_rt(double th, double tx, double ty, double q[4])
{
    /* real part: rotation by th about z; dual part: 1/2 t^ r with t^ the pure quaternion
     * (0, tx, ty, 0).  For a rotation about z and t in the plane, r has only (w, z) and
     * d only (x, y): the 4 components the footnote keeps. */
    double r[4] = {cos(th / 2.0), 0.0, 0.0, sin(th / 2.0)};
    double tq[4] = {0.0, tx, ty, 0.0};
    double d[4];
    qmul(tq, r, d);
    q[0] = r[0];
    q[1] = r[3];
    q[2] = 0.5 * d[1];
    q[3] = 0.5 * d[2];
}

void orc_rt_from_dq(const double q[4], double *th, double *tx, double *ty)
{
    /* t^ = 2 d r* for a unit real part */
    double r[4] = {q[0], 0.0, 0.0, q[1]};
    double rc[4] = {q[0], 0.0, 0.0, -q[1]};
    double d[4] = {0.0, q[2], q[3], 0.0};
    double tq[4];
    qmul(d, rc, tq);
    *th = 2.0 * atan2(r[3], r[0]);
    *tx = 2.0 * tq[1];
    *ty = 2.0 * tq[2];
}

void orc_apply_warp(double s, const double q[4], double px, double py, double out[2])
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1]);
    double qn[4] = {q[0] / n, q[1] / n, q[2] / n, q[3] / n};
    double th, tx, ty;
    orc_rt_from_dq(qn, &th, &tx, &ty);
    double c = cos(th), sn = sin(th);
    out[0] = s * (c * px - sn * py + tx);
    out[1] = s * (sn * px + c * py + ty);
}

/* Eqs. 2-4 at one point. Returns 0 and NaN output if the weights sum to 0. */
static int field_at(const double *q8, const double *c, const double *src, int n,
                    double px, double py, double alpha, double out[2])
{
    double sw = 0.0, ss = 0.0, sq[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i) {
        double dx = src[2 * i] - px, dy = src[2 * i + 1] - py;
        double w = c[i] * exp(-alpha * (dx * dx + dy * dy));
        sw += w;
        ss += w * q8[8 * i + 4];
        for (int k = 0; k < 4; ++k) sq[k] += w * q8[8 * i + k];
    }
    if (!(sw > 0.0) || !isfinite(sw)) {
        out[0] = out[1] = NAN;
        return 0;
    }
    double q[4] = {sq[0] / sw, sq[1] / sw, sq[2] / sw, sq[3] / sw};
    double xp[2];
    orc_apply_warp(ss / sw, q, px, py, xp);
    out[0] = xp[0] - px;
    out[1] = xp[1] - py;
    return 1;
}

int orc_field(const double *q8, const double *c, const double *src, int n,
              int gx0, int gy0, int gw, int gh, double alpha, double *disp, int nthreads)
{
    if (n < 0 || gw < 0 || gh < 0 || (n > 0 && (!q8 || !c || !src)) || !disp) return ORC_EINVAL;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int y = 0; y < gh; ++y)
        for (int x = 0; x < gw; ++x)
            field_at(q8, c, src, n, (double)(gx0 + x), (double)(gy0 + y), alpha,
                     disp + 2 * ((size_t)y * gw + x));
    return ORC_OK;
}

int orc_field_points(const double *q8, const double *c, const double *src, int n,
                     const double *pts, int npts, double alpha, double *disp, int nthreads)
{
    if (n < 0 || npts < 0 || !pts || !disp) return ORC_EINVAL;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int k = 0; k < npts; ++k)
        field_at(q8, c, src, n, pts[2 * k], pts[2 * k + 1], alpha, disp + 2 * k);
    return ORC_OK;
}

/* Eq. 8 at one point: min over the feature inliers j (the matches the fit keeps, c_j > 0)
 * of exp(beta d_j^2), written as the paper writes it (the exponential of every distance,
 * then the minimum); +inf when there is no inlier. */
static double uncertainty_at(const double *c, const double *src, int n, double px, double py,
                             double beta)
{
    double best = INFINITY;
    for (int j = 0; j < n; ++j) {
        if (!(c[j] > 0.0)) continue;
        double dx = src[2 * j] - px, dy = src[2 * j + 1] - py;
        double u = exp(beta * (dx * dx + dy * dy));
        if (u < best) best = u;
    }
    return best;
}

int orc_uncertainty(const double *c, const double *src, int n, int gx0, int gy0, int gw, int gh,
                    double beta, double *out, int nthreads)
{
    if (n < 0 || gw < 0 || gh < 0 || (n > 0 && (!c || !src)) || !out || !(beta > 0.0))
        return ORC_EINVAL;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int y = 0; y < gh; ++y)
        for (int x = 0; x < gw; ++x)
            out[(size_t)y * gw + x] =
                uncertainty_at(c, src, n, (double)(gx0 + x), (double)(gy0 + y), beta);
    return ORC_OK;
}

int orc_uncertainty_points(const double *c, const double *src, int n, const double *pts,
                           int npts, double beta, double *out, int nthreads)
{
    if (n < 0 || npts < 0 || (n > 0 && (!c || !src)) || !pts || !out || !(beta > 0.0))
        return ORC_EINVAL;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int k = 0; k < npts; ++k)
        out[k] = uncertainty_at(c, src, n, pts[2 * k], pts[2 * k + 1], beta);
    return ORC_OK;
}

/* Row (r_w, r_z, d_x, d_y, s, 1, 0, 0) of a similarity s (R(th) x + t), r_w >= 0. */
static void row_from_srt(double s, double th, double tx, double ty, double row[8])
{
    double q[4];
    orc_dq_from_rt(th, tx, ty, q);
    if (q[0] < 0.0)
        for (int k = 0; k < 4; ++k) q[k] = -q[k];
    for (int k = 0; k < 4; ++k) row[k] = q[k];
    row[4] = s;
    row[5] = 1.0;
    row[6] = row[7] = 0.0;
}

/* (s, th, t) of a row whose DQ part may be unnormalised (normalised by its real part). */
static void srt_from_row(const double row[8], double *s, double *th, double *tx, double *ty)
{
    double nr = sqrt(row[0] * row[0] + row[1] * row[1]);
    double q[4] = {row[0] / nr, row[1] / nr, row[2] / nr, row[3] / nr};
    orc_rt_from_dq(q, th, tx, ty);
    *s = row[4];
}

/* App. A: the updated warp of a node, (s_new, q_new) with s_new q_new(x) = ds dq(s_old q_old(x))
 * for every x: the two similarities composed -- scale ds s_old, rotation dth + th_old,
 * translation dR t_old + dt / s_old. */
void orc_compose(const double w_old[8], const double dw[8], double w_new[8])
{
    double so, tho, txo, tyo, ds, dth, dtx, dty;
    srt_from_row(w_old, &so, &tho, &txo, &tyo);
    srt_from_row(dw, &ds, &dth, &dtx, &dty);
    double c = cos(dth), sn = sin(dth);
    row_from_srt(ds * so, tho + dth, c * txo - sn * tyo + dtx / so, sn * txo + c * tyo + dty / so,
                 w_new);
}

/* Eqs. 2-3 at a point as a warp row (the blended DQ normalised by its real part, the blended
 * scale); returns 0 when the weights sum to 0. */
static int warp_at(const double *q8, const double *c, const double *src, int n, double px,
                   double py, double alpha, double row[8])
{
    double sw = 0.0, ss = 0.0, sq[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i) {
        double dx = src[2 * i] - px, dy = src[2 * i + 1] - py;
        double w = c[i] * exp(-alpha * (dx * dx + dy * dy));
        sw += w;
        ss += w * q8[8 * i + 4];
        for (int k = 0; k < 4; ++k) sq[k] += w * q8[8 * i + k];
    }
    if (!(sw > 0.0) || !isfinite(sw)) return 0;
    double nr = sqrt(sq[0] * sq[0] + sq[1] * sq[1]);
    for (int k = 0; k < 4; ++k) row[k] = sq[k] / nr;
    row[4] = ss / sw;
    row[5] = 1.0;
    row[6] = row[7] = 0.0;
    return 1;
}

/* Eq. 5 + App. A + Eq. 9 for every node i: its position at t-1, p = W_i,t-1(x_i,0); the
 * EMDQ warp dW at p (Eqs. 2-3 over the matches of t-1 -> t, positions src in frame t-1);
 * its uncertainty d_sigma^2 at p (Eq. 8); W_i,t = f(W_i,t-1, dW) (App. A) and
 * sigma^2_i,t = ds^2 sigma^2_i,t-1 + d_sigma^2 (Eq. 9).  A node where the field has no weight
 * keeps its warp and its uncertainty becomes +inf. */
int orc_node_track(const double *x0, const double *w_old, const double *s2_old, int nn,
                   const double *q8, const double *c, const double *src, int n, double alpha,
                   double beta, double *w_new, double *s2_new, int nthreads)
{
    if (nn < 0 || n < 0 || (nn > 0 && (!x0 || !w_old || !s2_old || !w_new || !s2_new)) ||
        (n > 0 && (!q8 || !c || !src)))
        return ORC_EINVAL;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int i = 0; i < nn; ++i) {
        const double *wo = w_old + 8 * (size_t)i;
        double so, th, tx, ty, p[2], dw[8];
        srt_from_row(wo, &so, &th, &tx, &ty);
        double qo[4] = {wo[0], wo[1], wo[2], wo[3]};
        double nr = sqrt(qo[0] * qo[0] + qo[1] * qo[1]);
        for (int k = 0; k < 4; ++k) qo[k] /= nr;
        orc_apply_warp(so, qo, x0[2 * i], x0[2 * i + 1], p);
        const double du = uncertainty_at(c, src, n, p[0], p[1], beta);
        if (!warp_at(q8, c, src, n, p[0], p[1], alpha, dw)) {
            for (int k = 0; k < 8; ++k) w_new[8 * (size_t)i + k] = wo[k];
            s2_new[i] = INFINITY;
            continue;
        }
        orc_compose(wo, dw, w_new + 8 * (size_t)i);
        s2_new[i] = dw[4] * dw[4] * s2_old[i] + du;
    }
    return ORC_OK;
}

/* Eqs. 12-15 for every node: eta = exp(-gamma |x_t - x_k|^2) with x_t = W_track(x_0) and
 * x_k = W_key(x_0) (Eq. 13); A = [[st^2, eta st sl], [eta st sl, sl^2]] (Eq. 12); the merged
 * uncertainty 1 / sum(A^-1) (Eq. 14) and the weights sigma_merge^2 A^-1 [1 1]^T (Eq. 15); the
 * merged warp is the weighted average of the two (DQ normalised by its real part, scale
 * averaged).  Where a weight is negative (or A is singular) the warp and uncertainty of the
 * smaller uncertainty are taken (ties: tracking). */
int orc_node_merge(const double *x0, const double *w_track, const double *s2_track,
                   const double *w_loop, const double *s2_loop, const double *w_key, int nn,
                   double gamma, double *w_out, double *s2_out)
{
    if (nn < 0 || (nn > 0 && (!x0 || !w_track || !s2_track || !w_loop || !s2_loop || !w_key ||
                              !w_out || !s2_out)))
        return ORC_EINVAL;
    for (int i = 0; i < nn; ++i) {
        const double *wt = w_track + 8 * (size_t)i, *wl = w_loop + 8 * (size_t)i,
                     *wk = w_key + 8 * (size_t)i;
        double s, th, tx, ty, qn[4], xt[2], xk[2];
        srt_from_row(wt, &s, &th, &tx, &ty);
        double nrt = sqrt(wt[0] * wt[0] + wt[1] * wt[1]);
        for (int k = 0; k < 4; ++k) qn[k] = wt[k] / nrt;
        orc_apply_warp(s, qn, x0[2 * i], x0[2 * i + 1], xt);
        srt_from_row(wk, &s, &th, &tx, &ty);
        double nrk = sqrt(wk[0] * wk[0] + wk[1] * wk[1]);
        for (int k = 0; k < 4; ++k) qn[k] = wk[k] / nrk;
        orc_apply_warp(s, qn, x0[2 * i], x0[2 * i + 1], xk);
        const double dx = xt[0] - xk[0], dy = xt[1] - xk[1];
        const double eta = exp(-gamma * (dx * dx + dy * dy));
        const double vt = s2_track[i], vl = s2_loop[i], st = sqrt(vt), sl = sqrt(vl);
        const double a01 = eta * st * sl, det = vt * vl - a01 * a01;
        /* A^-1 = [[vl, -a01], [-a01, vt]] / det */
        const double i00 = vl / det, i01 = -a01 / det, i11 = vt / det;
        const double sm = 1.0 / (i00 + 2.0 * i01 + i11);
        const double w0 = sm * (i00 + i01), w1 = sm * (i01 + i11);
        double *wo = w_out + 8 * (size_t)i;
        if (!(w0 >= 0.0) || !(w1 >= 0.0) || !isfinite(sm) || !isfinite(w0) || !isfinite(w1)) {
            const double *pick = vt <= vl ? wt : wl;
            for (int k = 0; k < 8; ++k) wo[k] = pick[k];
            s2_out[i] = vt <= vl ? vt : vl;
            continue;
        }
        double q[4];
        for (int k = 0; k < 4; ++k) q[k] = w0 * wt[k] / nrt + w1 * wl[k] / sqrt(wl[0] * wl[0] + wl[1] * wl[1]);
        double nq = sqrt(q[0] * q[0] + q[1] * q[1]);
        for (int k = 0; k < 4; ++k) wo[k] = q[k] / nq;
        wo[4] = w0 * wt[4] + w1 * wl[4];
        wo[5] = 1.0;
        wo[6] = wo[7] = 0.0;
        s2_out[i] = sm;
    }
    return ORC_OK;
}

/* Average of two warp rows with weights a, b (DQ normalised by its real part, scale averaged),
 * the reading of "weighted average" of warps used by Eqs. 15 and 22. */
static void average_rows(const double *wa, double a, const double *wb, double b, double *out)
{
    double na = sqrt(wa[0] * wa[0] + wa[1] * wa[1]), nb = sqrt(wb[0] * wb[0] + wb[1] * wb[1]);
    double q[4];
    for (int k = 0; k < 4; ++k) q[k] = a * wa[k] / na + b * wb[k] / nb;
    double nq = sqrt(q[0] * q[0] + q[1] * q[1]);
    for (int k = 0; k < 4; ++k) out[k] = q[k] / nq;
    out[4] = (a * wa[4] + b * wb[4]) / (a + b);
    out[5] = 1.0;
    out[6] = out[7] = 0.0;
}

static void apply_row(const double *w, double x, double y, double out[2])
{
    double nr = sqrt(w[0] * w[0] + w[1] * w[1]);
    double q[4] = {w[0] / nr, w[1] / nr, w[2] / nr, w[3] / nr};
    orc_apply_warp(w[4], q, x, y, out);
}

/* Sec. III-D, Eqs. 16-17 and ARAP1-3 as printed: the ARAP warp of every node i from the
 * motion x_j,0 -> x_j,t of all nodes j.  The columns of C_0 and C_t are
 * w_j^i (x_j,0 - x_i,0) and w_j^i (x_j,t - x_i,t), w_j^i = exp(-alpha |x_i,0 - x_j,0|^2):
 * centred on node i, the weight inside each column, no column dropped (the paper drops
 * columns of small weight only for speed).  ARAP1: R = U V^T from svd(C_t C_0^T), the det=+1
 * rotation, in 2-D the angle atan2(M10 - M01, M00 + M11) of M = C_t C_0^T.  ARAP2: s =
 * |vector(C_t)| / |vector(C_0)|.  ARAP3: t = the w-weighted average over j of
 * x_j,t / s - R x_j,0.  Then the quaternion from R and t.  Writes s[nn], th[nn], t[nn*2] and
 * q8[nn*8]; ORC_EDEGENERATE if some node has no spread. */
int orc_arap_fit(const double *x0, const double *xt, int nn, double alpha, double *s, double *th,
                 double *t, double *q8)
{
    if (nn < 1 || !x0 || !xt || !s || !th || !t || !q8) return ORC_EINVAL;
    int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(| : bad)
#endif
    for (int i = 0; i < nn; ++i) {
        double M[2][2] = {{0.0, 0.0}, {0.0, 0.0}};   /* C_t C_0^T */
        double n0 = 0.0, nt = 0.0;                    /* |vector(C_0)|^2, |vector(C_t)|^2 */
        for (int j = 0; j < nn; ++j) {
            double ex = x0[2 * j] - x0[2 * i], ey = x0[2 * j + 1] - x0[2 * i + 1];
            double w = exp(-alpha * (ex * ex + ey * ey));
            double c0[2] = {w * ex, w * ey};
            double ct[2] = {w * (xt[2 * j] - xt[2 * i]), w * (xt[2 * j + 1] - xt[2 * i + 1])};
            for (int r = 0; r < 2; ++r)
                for (int k = 0; k < 2; ++k) M[r][k] += ct[r] * c0[k];
            n0 += c0[0] * c0[0] + c0[1] * c0[1];
            nt += ct[0] * ct[0] + ct[1] * ct[1];
        }
        double ang = atan2(M[1][0] - M[0][1], M[0][0] + M[1][1]);     /* ARAP1 */
        double sc = sqrt(nt) / sqrt(n0);                             /* ARAP2 */
        double cr = cos(ang), sr = sin(ang);
        double W = 0.0, tx = 0.0, ty = 0.0;                          /* ARAP3 */
        for (int j = 0; j < nn; ++j) {
            double ex = x0[2 * j] - x0[2 * i], ey = x0[2 * j + 1] - x0[2 * i + 1];
            double w = exp(-alpha * (ex * ex + ey * ey));
            W += w;
            tx += w * (xt[2 * j] / sc - (cr * x0[2 * j] - sr * x0[2 * j + 1]));
            ty += w * (xt[2 * j + 1] / sc - (sr * x0[2 * j] + cr * x0[2 * j + 1]));
        }
        tx /= W;
        ty /= W;
        if (!(n0 > 0.0) || !isfinite(sc) || !isfinite(tx) || !isfinite(ty)) bad = 1;
        s[i] = sc;
        th[i] = ang;
        t[2 * i] = tx;
        t[2 * i + 1] = ty;
        double q[4];
        orc_dq_from_rt(ang, tx, ty, q);
        for (int k = 0; k < 4; ++k) q8[8 * i + k] = q[k];
        q8[8 * i + 4] = sc;
        q8[8 * i + 5] = 1.0;
        q8[8 * i + 6] = 0.0;
        q8[8 * i + 7] = 0.0;
    }
    return bad ? ORC_EDEGENERATE : ORC_OK;
}

/* Sec. III-D: ARAP smoothing of the merged node warps.  Iteration k: the nodes' positions
 * x_t = W^{k-1}(x_0) (W^0 = W_merge); the ARAP warp of every node from the nodes'
 * displacements x_0 -> x_t (orc_arap_fit); W^k = (W_merge + lambda W_ARAP) / (1 + lambda)
 * (Eq. 22), lambda = (1 + sigma_i^2) / (1 + 100); the cost of Eq. 21 summed over the nodes,
 * sum |W_merge(x_0) - W^k(x_0)|^2 + lambda |W_ARAP(x_0) - W^k(x_0)|^2.  Stops after max_iters
 * iterations or when the cost increases (keeping the previous warps). */
int orc_arap_smooth(const double *x0, const double *w_merge, const double *s2, int nn,
                    double alpha, int max_iters, double *w_out, double *costs)
{
    if (nn < 1 || !x0 || !w_merge || !s2 || !w_out || max_iters < 0) return ORC_EINVAL;
    double *xt = malloc(sizeof(double) * 2 * (size_t)nn);
    double *sc = malloc(sizeof(double) * (size_t)nn), *th = malloc(sizeof(double) * (size_t)nn);
    double *t = malloc(sizeof(double) * 2 * (size_t)nn), *wa = malloc(sizeof(double) * 8 * (size_t)nn);
    double *wk = malloc(sizeof(double) * 8 * (size_t)nn);
    if (!xt || !sc || !th || !t || !wa || !wk) {
        free(xt); free(sc); free(th); free(t); free(wa); free(wk);
        return ORC_EINVAL;
    }
    memcpy(w_out, w_merge, sizeof(double) * 8 * (size_t)nn);
    double prev = INFINITY;
    for (int k = 1; k <= max_iters; ++k) {
        for (int i = 0; i < nn; ++i) apply_row(w_out + 8 * (size_t)i, x0[2 * i], x0[2 * i + 1], xt + 2 * i);
        orc_arap_fit(x0, xt, nn, alpha, sc, th, t, wa);
        double cost = 0.0;
        for (int i = 0; i < nn; ++i) {
            const double lam = (1.0 + s2[i]) / (1.0 + 100.0);
            average_rows(w_merge + 8 * (size_t)i, 1.0, wa + 8 * (size_t)i, lam, wk + 8 * (size_t)i);
            double pm[2], pa[2], pk[2];
            apply_row(w_merge + 8 * (size_t)i, x0[2 * i], x0[2 * i + 1], pm);
            apply_row(wa + 8 * (size_t)i, x0[2 * i], x0[2 * i + 1], pa);
            apply_row(wk + 8 * (size_t)i, x0[2 * i], x0[2 * i + 1], pk);
            cost += (pm[0] - pk[0]) * (pm[0] - pk[0]) + (pm[1] - pk[1]) * (pm[1] - pk[1]) +
                    lam * ((pa[0] - pk[0]) * (pa[0] - pk[0]) + (pa[1] - pk[1]) * (pa[1] - pk[1]));
        }
        if (costs) costs[k - 1] = cost;
        if (cost > prev) break;
        prev = cost;
        memcpy(w_out, wk, sizeof(double) * 8 * (size_t)nn);
    }
    free(xt); free(sc); free(th); free(t); free(wa); free(wk);
    return ORC_OK;
}

/* Eq. 11 for every node: sigma_i^2 <- min(sigma_i^2, min_j (sigma_j^2 + exp(beta |x_i - y_j|^2)))
 * over the features j (positions y_j and uncertainties at the same time as the nodes' x_i). */
int orc_node_restrict(const double *x, const double *s2, int nn, const double *y,
                      const double *s2f, int m, double beta, double *s2_out)
{
    if (nn < 0 || m < 0 || (nn > 0 && (!x || !s2 || !s2_out)) || (m > 0 && (!y || !s2f)) ||
        !(beta > 0.0))
        return ORC_EINVAL;
    for (int i = 0; i < nn; ++i) {
        double best = s2[i];
        for (int j = 0; j < m; ++j) {
            double dx = x[2 * i] - y[2 * j], dy = x[2 * i + 1] - y[2 * j + 1];
            double b = s2f[j] + exp(beta * (dx * dx + dy * dy));
            if (b < best) best = b;
        }
        s2_out[i] = best;
    }
    return ORC_OK;
}

/* Eq. 6 for every key frame k: (1/N) sum_i |x_i,t - x_i,k| (xk: nk x nn x 2). */
int orc_keyframe_distances(const double *xt, const double *xk, int nn, int nk, double *out)
{
    if (nn < 1 || nk < 0 || !xt || (nk > 0 && (!xk || !out))) return ORC_EINVAL;
    for (int k = 0; k < nk; ++k) {
        double sum = 0.0;
        for (int i = 0; i < nn; ++i) {
            const double *p = xk + 2 * ((size_t)k * nn + i);
            sum += hypot(xt[2 * i] - p[0], xt[2 * i + 1] - p[1]);
        }
        out[k] = sum / nn;
    }
    return ORC_OK;
}

/* Eq. 10 for every feature j after the EMDQ t-1 -> t (rows q8, field weights c, positions src
 * in frame t-1 and dst in frame t): an inlier (c_j > 0) adds its squared error, sigma_j,EMDQ^2 =
 * |y_j - W_-j(x_j)|^2 with W_-j the field of the other inliers at x_j (Eqs. 2-3); an outlier
 * is propagated as Eq. 9 propagates a node, ds^2 sigma^2 + Eq. 8, with ds the field's scale at
 * x_j.  +inf where the field has no weight. */
int orc_feature_uncertainty(const double *src, const double *dst, int n, const double *q8,
                            const double *c, double alpha, double beta, const double *s2_prev,
                            double *s2_out)
{
    if (n < 1 || !src || !dst || !q8 || !c || !s2_prev || !s2_out || !(beta > 0.0))
        return ORC_EINVAL;
    double *e = malloc(sizeof(double) * (size_t)n);
    if (!e) return ORC_EINVAL;
    orc_residuals(src, dst, c, q8, n, alpha, e);
    for (int j = 0; j < n; ++j) {
        if (c[j] > 0.0) {
            s2_out[j] = s2_prev[j] + e[j];
            continue;
        }
        double row[8];
        if (!warp_at(q8, c, src, n, src[2 * j], src[2 * j + 1], alpha, row)) {
            s2_out[j] = INFINITY;
            continue;
        }
        s2_out[j] = row[4] * row[4] * s2_prev[j] +
                    uncertainty_at(c, src, n, src[2 * j], src[2 * j + 1], beta);
    }
    free(e);
    return ORC_OK;
}

/* Sec. III-E: the warps of new nodes at pts, the weighted average of the existing nodes' warps
 * (rows w at reference positions x0, weights exp(-alpha |p - x0_j|^2), the ARAP weights): the
 * Eqs. 2-3 blend with every weight 1.  NaN rows where the weights vanish. */
int orc_node_init(const double *x0, const double *w, int n, const double *pts, int npts,
                  double alpha, double *w_out)
{
    if (n < 1 || npts < 0 || !x0 || !w || (npts > 0 && (!pts || !w_out))) return ORC_EINVAL;
    double *ones = malloc(sizeof(double) * (size_t)n);
    if (!ones) return ORC_EINVAL;
    for (int j = 0; j < n; ++j) ones[j] = 1.0;
    for (int k = 0; k < npts; ++k)
        if (!warp_at(w, ones, x0, n, pts[2 * k], pts[2 * k + 1], alpha, w_out + 8 * (size_t)k))
            for (int m = 0; m < 8; ++m) w_out[8 * (size_t)k + m] = NAN;
    free(ones);
    return ORC_OK;
}

double orc_gamma_for_frame(int w, int h)
{
    double s = (w / 480.0 + h / 270.0) / 2.0;
    return 5e-3 / (s * s);
}

int orc_mstep(const double *src, const double *dst, const double *p, int n, double alpha,
              double *s, double *th, double *t, double *q8)
{
    if (n < 1 || !src || !dst || !p || !s || !th || !t || !q8) return ORC_EINVAL;
    int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(| : bad)
#endif
    for (int i = 0; i < n; ++i) {
        const double xi = src[2 * i], yi = src[2 * i + 1];
        /* weights w_j^i (Eq. 4 between matches, here times the inlier weight p_j) */
        double W = 0.0, xb[2] = {0.0, 0.0}, yb[2] = {0.0, 0.0};
        for (int j = 0; j < n; ++j) {
            double dx = src[2 * j] - xi, dy = src[2 * j + 1] - yi;
            double om = p[j] * exp(-alpha * (dx * dx + dy * dy));
            W += om;
            xb[0] += om * src[2 * j];
            xb[1] += om * src[2 * j + 1];
            yb[0] += om * dst[2 * j];
            yb[1] += om * dst[2 * j + 1];
        }
        double S[2][2] = {{0.0, 0.0}, {0.0, 0.0}};   /* C_t C_0^T */
        double vx = 0.0, vy = 0.0;                    /* |vector(C_0)|^2, |vector(C_t)|^2 */
        if (W > 0.0) {
            for (int k = 0; k < 2; ++k) { xb[k] /= W; yb[k] /= W; }
            for (int j = 0; j < n; ++j) {
                double dx = src[2 * j] - xi, dy = src[2 * j + 1] - yi;
                double om = p[j] * exp(-alpha * (dx * dx + dy * dy));
                double a0 = src[2 * j] - xb[0], a1 = src[2 * j + 1] - xb[1];
                double b0 = dst[2 * j] - yb[0], b1 = dst[2 * j + 1] - yb[1];
                S[0][0] += om * b0 * a0;
                S[0][1] += om * b0 * a1;
                S[1][0] += om * b1 * a0;
                S[1][1] += om * b1 * a1;
                vx += om * (a0 * a0 + a1 * a1);
                vy += om * (b0 * b0 + b1 * b1);
            }
        }
        /* Eq. 18: R = U V^T from svd(C_t C_0^T); in 2-D the rotation maximising
         * tr(R^T S) has angle atan2(S10 - S01, S00 + S11). */
        double ang = atan2(S[1][0] - S[0][1], S[0][0] + S[1][1]);
        /* Eq. 19: norm ratio */
        double sc = sqrt(vy / vx);
        /* Eq. 20: weighted average of X_t / s - R X_0 */
        double cr = cos(ang), sr = sin(ang);
        double tx = yb[0] / sc - (cr * xb[0] - sr * xb[1]);
        double ty = yb[1] / sc - (sr * xb[0] + cr * xb[1]);
        if (!(W > 0.0) || !(vx > 0.0) || !isfinite(sc) || !isfinite(tx) || !isfinite(ty))
            bad = 1;
        s[i] = sc;
        th[i] = ang;
        t[2 * i] = tx;
        t[2 * i + 1] = ty;
        double q[4];
        orc_dq_from_rt(ang, tx, ty, q);
        for (int k = 0; k < 4; ++k) q8[8 * i + k] = q[k];
        q8[8 * i + 4] = sc;
        q8[8 * i + 5] = 1.0;
        q8[8 * i + 6] = 0.0;
        q8[8 * i + 7] = 0.0;
    }
    return bad ? ORC_EDEGENERATE : ORC_OK;
}

int orc_residuals(const double *src, const double *dst, const double *p, const double *q8,
                  int n, double alpha, double *e)
{
    if (n < 1 || !src || !dst || !p || !q8 || !e) return ORC_EINVAL;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int j = 0; j < n; ++j) {
        const double xj = src[2 * j], yj = src[2 * j + 1];
        double sw = 0.0, ss = 0.0, sq[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < n; ++i) {
            if (i == j) continue;                    /* leave one out */
            double dx = src[2 * i] - xj, dy = src[2 * i + 1] - yj;
            double w = p[i] * exp(-alpha * (dx * dx + dy * dy));
            sw += w;
            ss += w * q8[8 * i + 4];
            for (int k = 0; k < 4; ++k) sq[k] += w * q8[8 * i + k];
        }
        if (!(sw > 0.0)) {
            e[j] = INFINITY;
            continue;
        }
        double q[4] = {sq[0] / sw, sq[1] / sw, sq[2] / sw, sq[3] / sw};
        double yh[2];
        orc_apply_warp(ss / sw, q, xj, yj, yh);
        double r0 = dst[2 * j] - yh[0], r1 = dst[2 * j + 1] - yh[1];
        e[j] = r0 * r0 + r1 * r1;
    }
    return ORC_OK;
}

static double sigma2_update(const double *p, const double *e, int n, double floor_)
{
    double num = 0.0, den = 0.0;
    for (int j = 0; j < n; ++j) {
        if (!isfinite(e[j])) continue;
        num += p[j] * e[j];
        den += p[j];
    }
    double s2 = den > 0.0 ? num / (2.0 * den) : floor_;
    return s2 > floor_ ? s2 : floor_;
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

int orc_fit(const double *src, const double *dst, int n, int frame_w, int frame_h,
            const orc_params *prm, const double *p0, double *q8, double *c, double *p,
            int *iters, double *sigma2, double *gamma, double *dp_trace)
{
    if (n < 3 || !src || !dst || !prm || !q8 || !c || !p || frame_w < 1 || frame_h < 1 ||
        prm->max_iters < 0)
        return ORC_EINVAL;
    const double alpha = prm->alpha > 0.0 ? prm->alpha : orc_alpha_for_frame(frame_w, frame_h);
    const double area = (double)frame_w * (double)frame_h;
    const double two_pi = 2.0 * acos(-1.0);
    double *s = malloc(sizeof(double) * n), *th = malloc(sizeof(double) * n);
    double *t = malloc(sizeof(double) * 2 * n), *e = malloc(sizeof(double) * n);
    double *pn = malloc(sizeof(double) * n);
    if (!s || !th || !t || !e || !pn) {
        free(s); free(th); free(t); free(e); free(pn);
        return ORC_EINVAL;
    }
    double g = 0.5;
    if (p0) {
        double m = 0.0;
        for (int j = 0; j < n; ++j) { p[j] = p0[j]; m += p0[j]; }
        g = clampd(m / n, 0.05, 0.95);
    } else {
        for (int j = 0; j < n; ++j) p[j] = 1.0;
    }
    /* step 0 */
    int rc = orc_mstep(src, dst, p, n, alpha, s, th, t, q8);
    orc_residuals(src, dst, p, q8, n, alpha, e);
    double s2 = sigma2_update(p, e, n, prm->sigma2_floor);
    int it = 0, converged = 0;
    while (rc == ORC_OK && it < prm->max_iters) {
        ++it;
        /* E-step: Gaussian inlier / uniform outlier posterior of each match */
        double dpmax = 0.0;
        for (int j = 0; j < n; ++j) {
            double G = isfinite(e[j]) ? exp(-e[j] / (2.0 * s2)) / (two_pi * s2) : 0.0;
            pn[j] = g * G / (g * G + (1.0 - g) / area);
            double d = fabs(pn[j] - p[j]);
            if (d > dpmax) dpmax = d;
        }
        memcpy(p, pn, sizeof(double) * n);
        /* M-step with the new weights, then the residuals and the mixture parameters */
        rc = orc_mstep(src, dst, p, n, alpha, s, th, t, q8);
        orc_residuals(src, dst, p, q8, n, alpha, e);
        s2 = sigma2_update(p, e, n, prm->sigma2_floor);
        double m = 0.0;
        for (int j = 0; j < n; ++j) m += p[j];
        g = clampd(m / n, 0.05, 0.95);
        if (dp_trace) dp_trace[it - 1] = dpmax;
        if (dpmax < prm->tol_p) { converged = 1; break; }
    }
    for (int j = 0; j < n; ++j) c[j] = p[j] >= 0.5 ? p[j] : 0.0;
    if (iters) *iters = it;
    if (sigma2) *sigma2 = s2;
    if (gamma) *gamma = g;
    free(s); free(th); free(t); free(e); free(pn);
    if (rc != ORC_OK) return rc;
    return converged ? ORC_OK : ORC_ENOCONV;
}

static double round_u8(double z)
{
    double r = floor(z + 0.5);
    return r < 0.0 ? 0.0 : (r > 255.0 ? 255.0 : r);
}

int orc_warp(const uint8_t *frame, int fw, int fh, int channels, int frame_pitch,
             const float *disp, int gx0, int gy0, int gw, int gh,
             uint8_t *canvas, int cw, int chh, int canvas_pitch, int ox, int oy)
{
    if (!frame || !disp || !canvas || fw < 1 || fh < 1 || (channels != 1 && channels != 3) ||
        gw < 0 || gh < 0 || frame_pitch < fw * channels || canvas_pitch < 4 * cw)
        return ORC_EINVAL;
    if (gw == 0 || gh == 0) return ORC_OK;
    if (gx0 + ox < 0 || gy0 + oy < 0 || gx0 + ox + gw > cw || gy0 + oy + gh > chh)
        return ORC_EINVAL;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int y = 0; y < gh; ++y) {
        for (int x = 0; x < gw; ++x) {
            const int px = gx0 + x, py = gy0 + y;
            const float *d = disp + 2 * ((size_t)y * gw + x);
            /* sample position in float32: the coverage and tap choices are integer
             * decisions, taken in the same precision as the kernel */
            volatile float ux = (float)px + d[0];
            volatile float uy = (float)py + d[1];
            double u0 = ux, u1 = uy;
            if (!(u0 >= 0.0 && u0 <= fw - 1.0 && u1 >= 0.0 && u1 <= fh - 1.0)) continue;
            int x0 = (int)floor(u0), y0 = (int)floor(u1);
            double fx = u0 - x0, fy = u1 - y0;
            int x1 = x0 + 1 < fw ? x0 + 1 : fw - 1;
            int y1 = y0 + 1 < fh ? y0 + 1 : fh - 1;
            uint8_t *cp = canvas + (size_t)(py + oy) * canvas_pitch + 4 * (size_t)(px + ox);
            double w = cp[3];
            for (int k = 0; k < channels; ++k) {
                double i00 = frame[(size_t)y0 * frame_pitch + (size_t)x0 * channels + k];
                double i10 = frame[(size_t)y0 * frame_pitch + (size_t)x1 * channels + k];
                double i01 = frame[(size_t)y1 * frame_pitch + (size_t)x0 * channels + k];
                double i11 = frame[(size_t)y1 * frame_pitch + (size_t)x1 * channels + k];
                double v = (1 - fx) * (1 - fy) * i00 + fx * (1 - fy) * i10 +
                           (1 - fx) * fy * i01 + fx * fy * i11;
                cp[k] = (uint8_t)round_u8((w * cp[k] + v) / (w + 1.0));
            }
            cp[3] = (uint8_t)(w + 1.0 < 30.0 ? w + 1.0 : 30.0);
        }
    }
    return ORC_OK;
}

int orc_insert_reference(const uint8_t *frame, int fw, int fh, int channels, int frame_pitch,
                         uint8_t *canvas, int cw, int chh, int canvas_pitch, int ox, int oy)
{
    if (!frame || !canvas || (channels != 1 && channels != 3) || ox < 0 || oy < 0 ||
        ox + fw > cw || oy + fh > chh || canvas_pitch < 4 * cw)
        return ORC_EINVAL;
    for (int y = 0; y < fh; ++y)
        for (int x = 0; x < fw; ++x) {
            uint8_t *cp = canvas + (size_t)(y + oy) * canvas_pitch + 4 * (size_t)(x + ox);
            for (int k = 0; k < channels; ++k)
                cp[k] = frame[(size_t)y * frame_pitch + (size_t)x * channels + k];
            cp[3] = 1;
        }
    return ORC_OK;
}
