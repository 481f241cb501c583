/*
 * FP64 CPU oracle for the EMDQ field + mosaic path of "Real-time Nonrigid Mosaicking of
 * Laparoscopy Images" (Zhou & Jayender).  TEST INFRASTRUCTURE ONLY: it is the reference the
 * CUDA path is checked against and the timed CPU baseline.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product library never does,
 * and the two share no code.
 *
 * Every routine is the plain definition written out, in double precision, following the
 * paper's equations; where the paper is silent the reading is stated beside the code.
 *
 * Conventions
 *   - Pixel coordinates, origin at the centre of reference pixel (0,0), x right, y down.
 *   - A warp function (Eq. 1) is a scale s and a planar dual quaternion q.  The planar DQ
 *     keeps the 4 non-zero components of the 8-D DQ (Sec. III footnote):
 *       q = (r_w, r_z, d_x, d_y),  r = (cos th/2, 0, 0, sin th/2),  d = 1/2 t^ (x) r.
 *   - Per-match rows are stored as 8 doubles: (r_w, r_z, d_x, d_y, s, 1, 0, 0).
 *   - Canvas pixels are 4 bytes (c0, c1, c2, weight); grey frames use c0 only.
 */
#ifndef EMDQ_ORACLE_H
#define EMDQ_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_EDEGENERATE = 2, ORC_ENOCONV = 3 };

typedef struct {
    double alpha;         /* Gaussian coefficient of Eq. 4; <= 0 -> derived (Sec. III-G) */
    int    max_iters;     /* EM iteration cap (reading: 20) */
    double tol_p;         /* stop when max_j |dp_j| < tol_p (reading: 1e-3) */
    double sigma2_floor;  /* lower bound of the residual variance (reading: 0.25 px^2) */
} orc_params;

/* Sec. III-G: alpha = 2e-4 / s^2 with s = (w/480 + h/270)/2. */
double orc_alpha_for_frame(int w, int h);
/* Sec. III-G: beta = 3e-3 / s^2, the coefficient of the uncertainty (Eq. 8). */
double orc_beta_for_frame(int w, int h);

/* Eq. 1 + footnote: planar DQ of the rigid part (R(th), t); inverse of the same. */
void orc_dq_from_rt(double th, double tx, double ty, double q[4]);
void orc_rt_from_dq(const double q[4], double *th, double *tx, double *ty);

/* Apply a (not necessarily unit) blended warp (s, q) to point p: normalise q by the norm
 * of its real part, recover (R, t), return s (R p + t).  Eq. 1 with Kavan-style DQB. */
void orc_apply_warp(double s, const double q[4], double px, double py, double out[2]);

/* Eqs. 2-4: dense displacement field on the grid [gx0, gx0+gw) x [gy0, gy0+gh).
 * q8: n rows of 8 (r_w, r_z, d_x, d_y, s, ...), c: per-match weight, src: n x 2 reference
 * positions.  disp: gh*gw*2 (dx, dy) row-major; NaN where sum of weights is 0. */
int orc_field(const double *q8, const double *c, const double *src, int n,
              int gx0, int gy0, int gw, int gh, double alpha, double *disp, int nthreads);

/* Same at arbitrary points pts (npts x 2). */
int orc_field_points(const double *q8, const double *c, const double *src, int n,
                     const double *pts, int npts, double alpha, double *disp, int nthreads);

/* EM M-step (reading of Eqs. 16-20): per match i, the p-weighted Gaussian similarity fit of
 * all matches j (including i).  Writes s[n], th[n], t[n*2] and q8[n*8].  Returns
 * ORC_EDEGENERATE if some row has no weight or no spread. */
/* Eq. 8: the uncertainty min_j exp(beta d_j^2) over the inliers (c_j > 0) at every pixel
 * of the window (out: gh x gw) or at npts points (pts: npts x 2); +inf without inliers. */
int orc_uncertainty(const double *c, const double *src, int n, int gx0, int gy0, int gw, int gh,
                    double beta, double *out, int nthreads);
int orc_uncertainty_points(const double *c, const double *src, int n, const double *pts,
                           int npts, double beta, double *out, int nthreads);
/* App. A: w_new (a warp row) with s_new q_new(x) = ds dq(s_old q_old(x)). */
void orc_compose(const double w_old[8], const double dw[8], double w_new[8]);
/* Eq. 5, App. A, Eq. 9: node warps and uncertainties after one tracking step (see the .c). */
int orc_node_track(const double *x0, const double *w_old, const double *s2_old, int nn,
                   const double *q8, const double *c, const double *src, int n, double alpha,
                   double beta, double *w_new, double *s2_new, int nthreads);
/* Eqs. 12-15: EKF merge of tracking and loop-closing node warps (see the .c). */
int orc_node_merge(const double *x0, const double *w_track, const double *s2_track,
                   const double *w_loop, const double *s2_loop, const double *w_key, int nn,
                   double gamma, double *w_out, double *s2_out);
/* Sec. III-D, Eqs. 16-17 and ARAP1-3 as printed: the ARAP warp of every node from the nodes'
 * motion x0 -> xt, with node-centred columns weighted inside (see the .c).  Writes s[nn],
 * th[nn], t[nn*2] and q8[nn*8]; ORC_EDEGENERATE if some node has no spread. */
int orc_arap_fit(const double *x0, const double *xt, int nn, double alpha, double *s, double *th,
                 double *t, double *q8);
/* Sec. III-D, Eqs. 21-22: ARAP smoothing of the node warps (see the .c); costs (max_iters,
 * may be NULL) receives the cost of every iteration run. */
int orc_arap_smooth(const double *x0, const double *w_merge, const double *s2, int nn,
                    double alpha, int max_iters, double *w_out, double *costs);
/* Sec. III-E: warps of new nodes, the weighted average of the existing nodes' (see the .c). */
int orc_node_init(const double *x0, const double *w, int n, const double *pts, int npts,
                  double alpha, double *w_out);
/* Eq. 10: feature uncertainties after one EMDQ (see the .c). */
int orc_feature_uncertainty(const double *src, const double *dst, int n, const double *q8,
                            const double *c, double alpha, double beta, const double *s2_prev,
                            double *s2_out);
/* Eq. 11: node uncertainties bounded by the features' (see the .c). */
int orc_node_restrict(const double *x, const double *s2, int nn, const double *y,
                      const double *s2f, int m, double beta, double *s2_out);
/* Eq. 6: mean node distance to every key frame (see the .c). */
int orc_keyframe_distances(const double *xt, const double *xk, int nn, int nk, double *out);
/* Sec. III-G: gamma = 5e-3 / s^2 (Eq. 13). */
double orc_gamma_for_frame(int w, int h);
int orc_mstep(const double *src, const double *dst, const double *p, int n, double alpha,
              double *s, double *th, double *t, double *q8);

/* EM leave-one-out residuals: e_j = |y_j - W_{-j}(x_j)|^2 where W_{-j} blends the warps of
 * all i != j with weights p_i exp(-alpha |x_i - x_j|^2).  e_j = +inf when that weight sum
 * is 0. */
int orc_residuals(const double *src, const double *dst, const double *p, const double *q8,
                  int n, double alpha, double *e);

/* Full EMDQ fit (reading of the absent EM definition, see header of emdq_oracle.c).
 * p0: initial inlier weights or NULL (all ones).  Outputs: q8 (n*8), c (n), p (n),
 * *iters, *sigma2, *gamma; dp_trace (max_iters doubles, may be NULL) receives max|dp|
 * of every iteration.  Returns ORC_OK, ORC_ENOCONV (cap reached, outputs valid),
 * ORC_EDEGENERATE or ORC_EINVAL. */
int orc_fit(const double *src, const double *dst, int n, int frame_w, int frame_h,
            const orc_params *prm, const double *p0, double *q8, double *c, double *p,
            int *iters, double *sigma2, double *gamma, double *dp_trace);

/* Eqs. 23-24 as read: gather warp + capped running-average blend of one frame into the
 * canvas over the window [gx0, gx0+gw) x [gy0, gy0+gh) of reference coordinates.
 * Canvas pixel of reference p is p + (ox, oy).  disp: gh*gw*2 float32 (the field as the
 * GPU stores it).  The sample position u = p + d is formed in float32 (the coverage and
 * tap decisions are integer decisions taken in the kernel's precision); interpolation and
 * blending are FP64. */
int orc_warp(const uint8_t *frame, int fw, int fh, int channels, int frame_pitch,
             const float *disp, int gx0, int gy0, int gw, int gh,
             uint8_t *canvas, int cw, int chh, int canvas_pitch, int ox, int oy);

/* Insert the reference frame at the canvas origin with weight 1 (Sec. III-F). */
int orc_insert_reference(const uint8_t *frame, int fw, int fh, int channels, int frame_pitch,
                         uint8_t *canvas, int cw, int chh, int canvas_pitch, int ox, int oy);

/* Threads the OpenMP build uses (1 without OpenMP). */
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
