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
 *
 * Readings (the paper is silent, garbled or delegates to its EMDQ reference)
 *   - Eq. 3 blends q without normalising it; a blended DQ is normalised by the norm of its
 *     real part before use (dual-quaternion blending).  In the planar case the real and
 *     dual parts are orthogonal, so that is the whole normalisation.
 *   - Eq. 18's C_0, C_t put the weight inside each column, centred on node i; the M-step
 *     here centres on the weighted centroids and applies each weight once (weighted least
 *     squares).  The rotation is the det=+1 solution, written in 2-D closed form.
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
