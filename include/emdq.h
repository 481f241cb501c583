/*
 * libemdq -- C ABI of the GB300 (sm_103a) EMDQ dense deformation field and mosaic warp of
 * "Real-time Nonrigid Mosaicking of Laparoscopy Images" (Zhou & Jayender).
 *
 * The three calls of the hot path, in the order a frame uses them:
 *   emdq_fit     feature matches -> per-match warp functions (scale + planar dual
 *                quaternion) and inlier weights                         (Sec. II, Eqs. 16-20)
 *   emdq_field   per-match warps -> dense displacement on a pixel grid   (Eqs. 1-4)
 *   mosaic_warp  frame + displacement -> blended into the mosaic canvas  (Sec. III-F, Eqs. 23-24)
 *
 * Common rules
 *   - Pointers documented "device" must be CUDA device (or managed) memory on the current
 *     device; "host" pointers are ordinary host memory.  The caller owns every buffer; the
 *     library never frees caller memory.  Scratch memory the kernels need is passed in as
 *     a caller-allocated workspace whose size the matching *_workspace_size() returns.
 *   - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 *     stream).  The return value reports argument errors and launch failures only;
 *     errors found on the device (non-finite input, degenerate fit, iteration cap, a
 *     bounded wait that gave up) are written to the device-side info record of the call
 *     and are visible after the stream is synchronised.
 *   - Coordinates are pixels with the origin at the centre of reference pixel (0, 0),
 *     x to the right, y down.  Points are stored as interleaved float pairs (x, y).
 *   - Warp rows are 8 floats: (r_w, r_z, d_x, d_y, s, 1, 0, 0) -- the real part
 *     (cos th/2, sin th/2), the dual part 1/2 t^ r reduced to its two non-zero components
 *     (the footnote to Eq. 1), the scale s of Eq. 1, a constant 1 and two zeros.
 *   - Canvas pixels are 4 bytes (c0, c1, c2, w): colour, and the merge weight of Eq. 24.
 *     Grey frames use c0 only.
 *
 * Thread safety: calls on different streams with disjoint outputs and workspaces may run
 * concurrently.  A workspace must not be shared by two calls in flight.
 */
#ifndef EMDQ_H
#define EMDQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EMDQ_ABI_VERSION 1

#if defined(__GNUC__)
#define EMDQ_API __attribute__((visibility("default")))
#else
#define EMDQ_API
#endif

typedef enum {
    EMDQ_OK = 0,
    EMDQ_EINVAL = 1,       /* bad argument: null pointer, size, layout, window off-canvas */
    EMDQ_EDEGENERATE = 2,  /* a fit row had no weight or no spread; no inlier weight left */
    EMDQ_ENOCONV = 3,      /* EM reached max_iters before max|dp| < tol_p; outputs valid */
    EMDQ_ETIMEOUT = 4,     /* a bounded device-side wait gave up (kernel returned early) */
    EMDQ_ECUDA = 5,        /* a CUDA runtime call failed (launch, attribute, memset) */
    EMDQ_EWORKSPACE = 6,   /* workspace null or smaller than *_workspace_size() */
    EMDQ_ENOTSUP = 7,      /* precision, size or device not supported by this build */
    EMDQ_ENONFINITE = 8    /* an input coordinate is NaN or infinite */
} emdq_status;

/* Field precisions. */
enum {
    EMDQ_FP32 = 0,  /* per-pixel direct sum on the CUDA cores, FP32 (the plain path) */
    EMDQ_BF16 = 1   /* separable Gaussian as tcgen05 GEMMs: BF16 operands, FP32 accumulate */
};

typedef struct {
    float alpha;         /* Eq. 4 coefficient (1/H^2); <= 0: derived from the frame size by
                            the rule of Sec. III-G, 2e-4 / s^2, s = (w/480 + h/270)/2 */
    int   max_iters;     /* EM iteration cap (default 20) */
    float tol_p;         /* EM stops when max_j |p_j - p_j,prev| < tol_p (default 1e-3) */
    float sigma2_floor;  /* lower bound of the residual variance, px^2 (default 0.25) */
    int   reserved[4];   /* zero, except for two settings of the fit's bounded device-side
                            waits (emdq_fit, emdq_fit_batch and the calls built on them):
                            [0] > 0 lowers the bound of every grid-barrier wait to that many
                            polls (default about 4 million, half a second; larger values keep
                            the default); [1] != 0 is a test of that bound: every barrier then
                            waits for one arrival more than the grid makes, no wait can end,
                            every CTA gives up after its bound and the fit's info record says
                            EMDQ_ETIMEOUT.  [2], [3]: zero. */
} emdq_params;

/* Device-side record a fit writes when it finishes (16 bytes, 4-byte aligned). */
typedef struct {
    int   status;        /* emdq_status of the device part of the fit */
    int   iters;         /* EM iterations run after step 0 */
    float sigma2;        /* final residual variance */
    float gamma;         /* final inlier fraction (mixing weight) */
} emdq_fit_info;

EMDQ_API void        emdq_default_params(emdq_params *prm);
/* Sec. III-G: alpha for a w x h frame. */
EMDQ_API float       emdq_alpha_for_frame(int w, int h);
/* Sec. III-G: beta (the coefficient of the uncertainty, Eq. 8) for a w x h frame, 3e-3 / s^2. */
EMDQ_API float       emdq_beta_for_frame(int w, int h);
EMDQ_API const char *emdq_status_string(int status);
EMDQ_API int         emdq_abi_version(void);

/* ------------------------------------------------------------------ emdq_fit ---------
 * EMDQ mismatch removal and per-match warp estimation (Sec. II: "the input of EMDQ is the
 * coordinates of image feature matches").  The paper delegates the EM iteration to its
 * EMDQ reference; this library implements the reading documented with the oracle:
 *   step 0    p = p0 (or 1); M-step; leave-one-out residuals; sigma^2; gamma = 1/2
 *   iterate   E-step: p_j = gamma G_j / (gamma G_j + (1-gamma)/(w h)),
 *               G_j = exp(-e_j / (2 sigma^2)) / (2 pi sigma^2)
 *             M-step: per match i the closed-form similarity of Eqs. 18-20 fitted to all
 *               matches with weights p_j exp(-alpha |x_i - x_j|^2) (moments taken about
 *               the weighted centroid -- found by a first pass at step 0, the previous
 *               round's afterwards -- so FP32 sums do not cancel)
 *             residuals e_j = |y_j - W_{-j}(x_j)|^2 of the leave-one-out blend (Eqs. 2-4)
 *             sigma^2 = max(sum p e / (2 sum p), floor), gamma = clamp(mean p, .05, .95)
 *   output    q_out rows, c_out[i] = p_i if p_i >= 1/2 else 0, p_out = p
 *
 *   src, dst   device, n x 2 float: match positions in the reference frame and frame t
 *   n          3 <= n <= emdq_fit_max_n()
 *   frame_w/h  size of frame t (outlier density 1/(w h); alpha rule)
 *   prm        host; NULL = defaults
 *   p0         device, n float initial inlier weights in [0, 1], or NULL for all ones
 *              (a negative or non-finite weight gives info->status = EMDQ_ENONFINITE)
 *   q_out      device, n x 8 float warp rows (written)
 *   c_out      device, n float field weights (written)
 *   p_out      device, n float final posteriors (written), may be NULL
 *   info       device emdq_fit_info (written)
 *   workspace  device scratch of emdq_fit_workspace_size(n) bytes, 256-byte aligned
 * Returns EMDQ_EINVAL / EMDQ_EWORKSPACE / EMDQ_ENOTSUP / EMDQ_ECUDA on the host; the
 * device outcome (OK, ENOCONV, EDEGENERATE, ETIMEOUT, ENONFINITE) is in info->status.
 */
EMDQ_API int         emdq_fit_max_n(void);
EMDQ_API size_t      emdq_fit_workspace_size(int n);
EMDQ_API emdq_status emdq_fit(const float *src, const float *dst, int n, int frame_w, int frame_h,
                     const emdq_params *prm, const float *p0, float *q_out, float *c_out,
                     float *p_out, emdq_fit_info *info, void *workspace,
                     size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ emdq_fit_batch ---
 * Many independent fits (frames of a sequence, pairs of different sizes) in one
 * cooperative launch: each problem runs the emdq_fit iteration on its own group of CTAs
 * with its own barrier, so the latency-bound EM rounds of several fits overlap on the GPU.
 * Results are those of calling emdq_fit on each problem.
 *
 *   problems   host array of `count` descriptors (1 <= count <= 64); every pointer in a
 *              descriptor follows the rules of the matching emdq_fit argument
 *   workspace  device scratch of emdq_fit_batch_workspace_size(problems, count) bytes,
 *              256-byte aligned
 * Returns EMDQ_ENOTSUP when count exceeds 64 or a problem exceeds emdq_fit_max_n().
 */
typedef struct {
    const float *src, *dst;     /* device, n x 2 float */
    int n, frame_w, frame_h;
    const float *p0;            /* device, n float, or NULL */
    float *q_out, *c_out;       /* device, n x 8 and n float (written) */
    float *p_out;               /* device, n float (written) or NULL */
    emdq_fit_info *info;        /* device (written) */
} emdq_fit_problem;

EMDQ_API size_t      emdq_fit_batch_workspace_size(const emdq_fit_problem *problems, int count);
/* CTAs are split over the problems in proportion to n^2 (the EM work per round), at least
 * one and at most ceil(n / 8) each. */
EMDQ_API emdq_status emdq_fit_batch(const emdq_fit_problem *problems, int count,
                                    const emdq_params *prm, void *workspace,
                                    size_t workspace_bytes, void *stream);

/* The batch launch with an explicit split: problem b runs on ctas[b] CTAs (host array of
 * `count` ints, each >= 1, summing to at most emdq_fit_batch_capacity(problems, count);
 * otherwise EMDQ_EINVAL).  ctas = NULL is emdq_fit_batch.  Results depend on the split only
 * through FP32 rounding: the summation order of the sigma^2 partial sums and the M-step's
 * groups of rows (each CTA groups its own range of rows). */
EMDQ_API emdq_status emdq_fit_batch_ex(const emdq_fit_problem *problems, int count,
                                       const emdq_params *prm, const int *ctas, void *workspace,
                                       size_t workspace_bytes, void *stream);

/* The batch in phases, for batches whose fits need very different numbers of EM rounds (one
 * slow fit otherwise holds the whole launch while the CTAs of the others idle).  Phase 1 is
 * emdq_fit_batch with max_iters = phase_iters[0].  Each later phase k is one more cooperative
 * launch in which the fits that ran phase_iters[k-1] rounds without converging (status
 * EMDQ_ENOCONV) take every CTA, split on the device in proportion to n^2, and continue for at
 * most phase_iters[k] - phase_iters[k-1] more rounds from the state their last round left (the
 * posteriors p_out, sigma^2 and gamma of the fit record, the order, centroids and residuals in
 * the workspace): the same iteration as one launch, with the FP32 roundings of the new split
 * (the M-step's row groups, the sigma^2 partial sums).  Finished fits are left as they are.
 * info->iters counts every phase's rounds; phase_iters[nphases - 1] takes the place of
 * prm->max_iters.  The workspace must not change between the phases (it is one call).
 *
 *   phase_iters  host, nphases (1..16) strictly increasing round counts >= 1
 *   problems     as emdq_fit_batch; every p_out must be non-NULL (EMDQ_EINVAL otherwise)
 *   workspace    as emdq_fit_batch (the same size)
 * Asynchronous on `stream`, all phases on the device (no host synchronisation between them). */
EMDQ_API emdq_status emdq_fit_batch_phases(const emdq_fit_problem *problems, int count,
                                           const emdq_params *prm, const int *phase_iters,
                                           int nphases, void *workspace, size_t workspace_bytes,
                                           void *stream);

/* CTAs of the batch kernel that are co-resident on the current device for these problems
 * (the largest n sets the shared memory per CTA); 0 on error. */
EMDQ_API int         emdq_fit_batch_capacity(const emdq_fit_problem *problems, int count);

/* Autotuner of the batch split (not in the paper: a launch-configuration search).  Runs
 * the batch with CTAs split in proportion to n^e for e in {0, 1, 1.5, 2, 2.5, 3}, each once
 * untimed and then `reps` times (1..100) timed with CUDA events on `stream`, and writes the
 * fastest split to ctas_out (host, count ints) and its best time in ms to ms_out (host,
 * may be NULL).  Synchronises the stream; refuses (EMDQ_EINVAL) while the stream is being
 * captured.  The problems' outputs hold the last run's results. */
EMDQ_API emdq_status emdq_fit_batch_autotune(const emdq_fit_problem *problems, int count,
                                             const emdq_params *prm, void *workspace,
                                             size_t workspace_bytes, void *stream, int reps,
                                             int *ctas_out, float *ms_out);

/* ------------------------------------------------------------------ emdq_fit_noalloc -
 * emdq_fit for callers that cannot allocate device memory.  The paper has no counterpart:
 * this is a deployment variant.  Some callers must not call cudaMalloc once they are
 * running -- a real-time video loop (cudaMalloc can stall the whole device while it
 * runs), a plug-in inside a host application that owns every device allocation through
 * its own pool, or a service whose memory is fixed at start-up -- and so cannot provide
 * the workspace emdq_fit asks for.  This entry point takes the same inputs and outputs
 * (all still allocated by the caller) and keeps its scratch in a fixed array of about
 * 136 KB inside the library, which every GPU that loads the library holds until exit.
 *
 *   - n must be at most 5120 (emdq_fit_max_n()); larger n returns EMDQ_ENOTSUP.
 *   - It allocates nothing and calls no allocating routine.  Its first call on each device
 *     looks up the array's device address once (cudaGetSymbolAddress, with that device
 *     current); make that first call before any stream capture.
 *   - Every call shares the one array, which keeps the previous call's contents (the
 *     parts that must start at zero are cleared on the call's stream).  Calls that can
 *     overlap on the GPU -- on different streams, or on different host threads -- race on
 *     that array: serialise them (for example, issue them all on one stream).
 * Arguments, results and errors are those of emdq_fit.
 */
EMDQ_API emdq_status emdq_fit_noalloc(const float *src, const float *dst, int n, int frame_w,
                             int frame_h, const emdq_params *prm, const float *p0,
                             float *q_out, float *c_out, float *p_out, emdq_fit_info *info,
                             void *stream);

/* ------------------------------------------------------------------ emdq_field -------
 * Dense displacement field (Eqs. 2-4 with Eq. 1): for every pixel p of the grid
 * [grid_x0, grid_x0 + grid_w) x [grid_y0, grid_y0 + grid_h) (reference coordinates),
 *   w_i = c_i exp(-alpha |x_i - p|^2),  s_p = sum w_i s_i / sum w_i,
 *   q_p = sum w_i q_i / sum w_i normalised by |(r_w, r_z)|,
 *   disp(p) = s_p (R(q_p) p + t(q_p)) - p.
 * Pixels where sum w_i = 0 get NaN.
 *
 *   q, c, src  device: n x 8 warp rows, n weights, n x 2 reference positions (the fit's
 *              outputs and its src)
 *   alpha      > 0
 *   precision  EMDQ_FP32 or EMDQ_BF16
 *   disp_out   device, grid_h x grid_w x 2 float, row-major (written)
 *   workspace  device scratch of emdq_field_workspace_size(...) bytes (may be 0 bytes for
 *              EMDQ_FP32), 256-byte aligned
 */
EMDQ_API size_t      emdq_field_workspace_size(int n, int grid_w, int grid_h, int precision);
EMDQ_API emdq_status emdq_field(const float *q, const float *c, const float *src, int n,
                       int grid_x0, int grid_y0, int grid_w, int grid_h, float alpha,
                       int precision, float *disp_out, void *workspace,
                       size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ emdq_field_batch --
 * Several BF16 fields -- the frames of a sequence or the pairs of a batch -- in one
 * operand-preparation launch and one persistent tensor-core launch that walks the tiles of
 * every field in turn, so the fixed cost of the two launches is paid once per batch.  Each
 * field is exactly what emdq_field with EMDQ_BF16 computes for the same arguments.
 *
 *   problems   host array of `count` descriptors (1 <= count <= 16); the pointers follow the
 *              rules of the matching emdq_field arguments
 *   workspace  device scratch of emdq_field_batch_workspace_size(problems, count) bytes,
 *              256-byte aligned, not shared with a call in flight
 * Returns EMDQ_EINVAL for a bad descriptor, EMDQ_ENOTSUP for count > 16 or a device without
 * tcgen05, EMDQ_EWORKSPACE / EMDQ_ECUDA as emdq_field.
 */
typedef struct {
    const float *q;             /* device, n x 8 warp rows (emdq_fit's q_out) */
    const float *c;             /* device, n field weights (emdq_fit's c_out) */
    const float *src;           /* device, n x 2 match positions in the reference frame */
    int n;
    int grid_x0, grid_y0, grid_w, grid_h;   /* the pixel window, reference coordinates */
    float alpha;                /* Gaussian weight exp(-alpha |p - x_i|^2) */
    float *disp_out;            /* device, grid_h x grid_w x 2 float (written) */
} emdq_field_problem;

EMDQ_API size_t      emdq_field_batch_workspace_size(const emdq_field_problem *problems, int count);
EMDQ_API emdq_status emdq_field_batch(const emdq_field_problem *problems, int count,
                                      void *workspace, size_t workspace_bytes, void *stream);

/* Tile shape of the batched field (no counterpart in the paper: a launch configuration).  The
 * tensor-core GEMM covers each window in tiles of 128 pixels x `tile_rows` pixel rows (the MMA
 * computes all six blend sums of the tile's rows at once, N = 6 tile_rows); tile_rows is one
 * of 16, 24, 32 (the default) and 40.  Every tile height gives the same field bits (each
 * output's accumulation over the matches is the same); it changes only the speed: taller
 * tiles carry more multiply-adds per operand byte and per MMA, shorter ones make more tiles
 * for windows too small to occupy every SM.
 *   emdq_field_batch_ex        emdq_field_batch with an explicit tile height (EMDQ_ENOTSUP
 *                              for another value); the same workspace size
 *   emdq_field_batch_tile_rows the tile height emdq_field_batch uses for such a batch: the
 *                              one the autotuner recorded for its size class (the mean window
 *                              size and mean match count, each to a power of two, and the
 *                              field count), else 32; -1 for bad arguments
 *   emdq_field_batch_autotune  times every tile height on this batch (one untimed call, then
 *                              `reps` calls each, CUDA events on `stream`; synchronises the
 *                              stream), records the fastest for the batch's size class, and
 *                              returns it in *tile_rows_out with its time per call in *ms_out
 *                              (either may be NULL).  The outputs hold the last call's field.
 *                              The record is per process and host-thread-safe.
 */
EMDQ_API emdq_status emdq_field_batch_ex(const emdq_field_problem *problems, int count,
                                         int tile_rows, void *workspace, size_t workspace_bytes,
                                         void *stream);
EMDQ_API int         emdq_field_batch_tile_rows(const emdq_field_problem *problems, int count);
EMDQ_API emdq_status emdq_field_batch_autotune(const emdq_field_problem *problems, int count,
                                               void *workspace, size_t workspace_bytes,
                                               void *stream, int reps, int *tile_rows_out,
                                               float *ms_out);

/* ------------------------------------------------------------------ emdq_uncertainty -
 * Uncertainty of the EMDQ field (Sec. III-C, Eq. 8): at every pixel p of the window
 * (reference coordinates, as emdq_field), the minimum over the feature inliers j (the
 * matches the fit keeps: c_j > 0) of exp(beta |p - x_j|^2), i.e. exp(beta d^2) with d the
 * distance to the nearest inlier.  Low near inliers, growing fast away from them; +inf where
 * beta d^2 exceeds the FP32 range or when there is no inlier.
 *
 *   c, src     device, n field weights (emdq_fit's c_out) and n x 2 match positions in the
 *              reference frame (8-byte aligned); may be NULL when n = 0
 *   grid_*     the pixel window
 *   beta       > 0 (emdq_beta_for_frame gives the paper's value for a frame size)
 *   out        device, grid_h x grid_w float (written)
 * Returns EMDQ_EINVAL for bad arguments, EMDQ_ENOTSUP for a window taller than 524,280 rows
 * (65535 tiles of 8 rows); an empty window writes nothing.
 */
EMDQ_API emdq_status emdq_uncertainty(const float *c, const float *src, int n, int grid_x0,
                                      int grid_y0, int grid_w, int grid_h, float beta, float *out,
                                      void *stream);

/* ------------------------------------------------------------------ deformation nodes -
 * The SLAM state the field is carried on (Sec. III-A): nodes i with reference positions x_i,0
 * and warp rows W_i (r_w, r_z, d_x, d_y, s, 1, 0, 0; the node's position at t is W_i(x_i,0))
 * and uncertainties sigma_i^2.
 *
 * Common to emdq_node_track, emdq_node_merge, emdq_node_restrict, emdq_keyframe_distances,
 * emdq_feature_uncertainty and emdq_node_init: every array is a caller-owned device buffer
 * (positions nx2 float, 8-byte aligned; warp rows nx8 float, 16-byte aligned where a fit's q is
 * taken) and the library allocates nothing; the call is asynchronous on `stream` and outputs may
 * not alias inputs.  EMDQ_EINVAL, before any launch: a negative count, a coefficient (alpha,
 * beta, gamma) that is not positive and finite, or a missing or misaligned array the call needs
 * (emdq_keyframe_distances also needs nn >= 1, emdq_node_init nn >= 1).  A count of 0 for what
 * is written (nodes, features, key frames, points) returns EMDQ_OK without work.  EMDQ_ECUDA if
 * the launch fails.
 *
 * emdq_node_track (Eq. 5, App. A, Eq. 9): for every node, p = W_i,t-1(x_i,0); dW = the Eqs. 2-3
 * blend at p of the t-1 -> t fit (q, c, src as emdq_field takes them; src in frame t-1);
 * W_i,t = f(W_i,t-1, dW), the warp with s_new q_new(x) = ds dq(s_old q_old(x)) (App. A);
 * sigma_i,t^2 = ds^2 sigma_i,t-1^2 + min over the inliers of exp(beta |p - x_j|^2) (Eqs. 9, 8).
 * A node where the field has no weight keeps its warp and gets sigma^2 = +inf.
 *   x0        device, nn x 2 float (8-byte aligned); w_old, w_new: nn x 8 float; s2_*: nn float
 *   alpha, beta > 0 (emdq_alpha_for_frame, emdq_beta_for_frame)
 *
 * emdq_node_merge (Eqs. 12-15): for every node, eta = exp(-gamma |x_t - x_k|^2) with x_t =
 * W_track(x0), x_k = W_key(x0) (the node at the loop-closing key frame); A = [[st^2, eta st sl],
 * [eta st sl, sl^2]]; sigma^2 = 1 / sum(A^-1); weights sigma^2 A^-1 [1 1]^T; the merged warp is
 * the weighted average (DQ normalised by its real part, scale averaged).  Where a weight is
 * negative the warp and uncertainty of the smaller uncertainty are taken (ties: tracking).
 *   gamma > 0 (emdq_gamma_for_frame); w_out, s2_out may not alias the inputs
 */
EMDQ_API float       emdq_gamma_for_frame(int w, int h);
EMDQ_API emdq_status emdq_node_track(const float *x0, const float *w_old, const float *s2_old,
                                     int nn, const float *q, const float *c, const float *src,
                                     int n, float alpha, float beta, float *w_new, float *s2_new,
                                     void *stream);
EMDQ_API emdq_status emdq_node_merge(const float *x0, const float *w_track, const float *s2_track,
                                     const float *w_loop, const float *s2_loop, const float *w_key,
                                     int nn, float gamma, float *w_out, float *s2_out,
                                     void *stream);

/* emdq_node_restrict (Eq. 11): s2_out_i = min(s2_i, min_j (s2f_j + exp(beta |x_i - y_j|^2))), the
 * node uncertainties bounded by the features' (node positions x and feature positions y at the
 * same time; nn x 2 and m x 2 float, 8-byte aligned).
 * emdq_keyframe_distances (Eq. 6): out_k = (1/N) sum_i |xt_i - xk_k,i| for nk key frames (xk:
 * nk x nn x 2 float, the nodes' positions at each key frame); the caller adds frame t as a key
 * frame when the smallest of them exceeds its threshold H.
 */
/* emdq_feature_uncertainty (Eq. 10): after the EMDQ t-1 -> t (q, c, src as emdq_field takes
 * them, dst the matches' positions in frame t), s2_out_j = s2_prev_j + |y_j - W_-j(x_j)|^2 for an
 * inlier (c_j > 0; W_-j the field of the other inliers at x_j), and ds^2 s2_prev_j + Eq. 8 at x_j
 * for an outlier (ds the field's scale there, as Eq. 9 propagates a node); +inf where the field
 * has no weight.  The caller keeps the features' identities across frames.
 */
EMDQ_API emdq_status emdq_feature_uncertainty(const float *src, const float *dst, int n,
                                              const float *q, const float *c, float alpha,
                                              float beta, const float *s2_prev, float *s2_out,
                                              void *stream);
EMDQ_API emdq_status emdq_node_restrict(const float *x, const float *s2, int nn, const float *y,
                                        const float *s2f, int m, float beta, float *s2_out,
                                        void *stream);
EMDQ_API emdq_status emdq_keyframe_distances(const float *xt, const float *xk, int nn, int nk,
                                             float *out, void *stream);

/* Node insertion (Sec. III-E).  emdq_hex_nodes (host, no GPU): the nodes of a w x h frame, the
 * hexagonal lattice with the given spacing through the image centre ((w-1)/2, (h-1)/2; rows
 * spacing*sqrt(3)/2 apart, alternate rows shifted by spacing/2) grown breadth-first from the
 * centre over every node's 6 neighbours, keeping the points within the lattice's covering radius
 * spacing/sqrt(3) of the frame, so every pixel has a node within that radius.  Writes up to
 * `capacity` positions (x, y) to the host array x0_out in that order and returns how many there
 * are (-1 for bad arguments).
 * emdq_node_init: the warps of new nodes at pts (npts x 2, device), each the weighted average
 * of the existing nodes' warps w (nn x 8 at reference positions x0, nn x 2) with the ARAP weights
 * exp(-alpha |p - x0_j|^2) -- the Eqs. 2-3 blend with every weight 1; NaN rows where every
 * weight vanishes.
 */
EMDQ_API int         emdq_hex_nodes(int w, int h, float spacing, float *x0_out, int capacity);
EMDQ_API emdq_status emdq_node_init(const float *x0, const float *w, int nn, const float *pts,
                                    int npts, float alpha, float *w_out, void *stream);

/* emdq_arap_smooth (Sec. III-D, Eqs. 16-17, ARAP1-3, 21-22): ARAP smoothing of the merged node
 * warps.  At most max_iters iterations (the paper uses 5) of: positions x_t = W(x_0); the ARAP
 * warp of every node i as printed -- C_0 and C_t with the columns w_j (x_j,0 - x_i,0) and
 * w_j (x_j,t - x_i,t) over every node j, w_j = exp(-alpha |x_i,0 - x_j,0|^2), rotation U V^T of
 * svd(C_t C_0^T) (the det = +1 solution), scale |C_t| / |C_0|, translation the w-weighted average
 * of x_j,t / s - R x_j,0 (a node whose columns all vanish keeps its current warp as its ARAP
 * warp); W = (W_merge + lambda W_ARAP) / (1 + lambda) with lambda = (1 + sigma_i^2) / 101;
 * stopping, with the previous warps kept, when the summed cost of Eq. 21 rises.  Runs on the
 * stream without host synchronisation.
 *   x0        device, nn x 2 float (8-byte aligned), 3 <= nn <= 2^22
 *   w_merge   device, nn x 8 float warp rows; s2: device, nn float merged uncertainties
 *   w_out     device, nn x 8 float (16-byte aligned; written), not aliasing w_merge
 *   workspace device, emdq_arap_workspace_size(nn) bytes, 256-byte aligned
 * Returns EMDQ_EINVAL for bad arguments, EMDQ_ENOTSUP above 2^22 nodes, EMDQ_EWORKSPACE for a
 * missing, short or misaligned workspace (all before any launch), and EMDQ_ECUDA if a copy or
 * launch fails.
 */
EMDQ_API size_t      emdq_arap_workspace_size(int nn);
EMDQ_API emdq_status emdq_arap_smooth(const float *x0, const float *w_merge, const float *s2,
                                      int nn, float alpha, int max_iters, float *w_out,
                                      void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ mosaic_warp ------
 * Gather warp + capped running-average blend of frame t into the canvas (Sec. III-F,
 * Eqs. 23-24 as read: the paper's printed blend lacks its normalisation and its cap reads
 * max{w+1, 30}).  For every grid pixel p (reference coordinates), u = p + disp(p) is
 * formed in FP32; if 0 <= u_x <= fw-1 and 0 <= u_y <= fh-1 the frame is sampled
 * bilinearly at u and canvas pixel P = p + (origin_x, origin_y) is updated
 *   c <- clamp(floor((w c + v)/(w + 1) + 1/2), 0, 255),  w <- min(w + 1, 30)
 * otherwise the canvas pixel is left untouched (also for NaN displacements).
 *
 *   frame        device, fh rows of frame_pitch bytes, pixels of `channels` bytes (1 or 3)
 *   disp         device, grid_h x grid_w x 2 float (emdq_field's output)
 *   canvas       device, canvas_h rows of canvas_pitch bytes (multiple of 4, >= 4 canvas_w),
 *                4-byte pixels, 4-byte aligned
 *   origin_x/y   canvas position of reference pixel (0, 0)
 * The grid, shifted by the origin, must lie inside the canvas (else EMDQ_EINVAL); a frame of
 * fh x frame_pitch bytes must hold fewer than 2^31 bytes (else EMDQ_ENOTSUP).
 */
EMDQ_API emdq_status mosaic_warp(const uint8_t *frame, int fw, int fh, int channels, int frame_pitch,
                        const float *disp, int grid_x0, int grid_y0, int grid_w, int grid_h,
                        uint8_t *canvas, int canvas_w, int canvas_h, int canvas_pitch,
                        int origin_x, int origin_y, void *stream);

/* ------------------------------------------------------------------ mosaic_warp_batch -
 * Up to 8 frames of one sequence (same size, channels and pitch) blended into one canvas in
 * one launch: canvas pixels are taken through the frames in array order, exactly as the
 * same mosaic_warp calls in that order would leave them (a pixel's update depends only on
 * its own earlier updates), with the canvas read and written once per pixel and the loads
 * of all the frames in flight together.  Each frame has its own field and window (the rules
 * of mosaic_warp's frame, disp and grid arguments); an empty window is skipped.
 * Returns EMDQ_ENOTSUP for count > 8, otherwise the errors of mosaic_warp.
 */
typedef struct {
    const uint8_t *frame;       /* device, fh rows of frame_pitch bytes */
    const float *disp;          /* device, grid_h x grid_w x 2 float */
    int grid_x0, grid_y0, grid_w, grid_h;
} mosaic_frame;

EMDQ_API emdq_status mosaic_warp_batch(const mosaic_frame *frames, int count, int fw, int fh,
                                       int channels, int frame_pitch, uint8_t *canvas,
                                       int canvas_w, int canvas_h, int canvas_pitch, int origin_x,
                                       int origin_y, void *stream);

/* ------------------------------------------------------------------ emdq_batch -------
 * The whole path for a batch of independent pairs in one call (not in the paper: a
 * batching front end).  On `stream`, in order: the learned warm start of every pair (when
 * warm_params is not NULL; else plain EM from p = 1), all EMDQ fits in one cooperative
 * launch (CTAs split per fit_ctas, or in proportion to n^2 when it is NULL), then per group
 * of up to 16 pairs their BF16 fields and warps fused in one emdq_mosaic_pairs call, or,
 * where two pairs of the group update overlapping canvas rows or differ in channels (or the
 * fused call refuses the group), one emdq_field_batch call followed by the warps of its pairs
 * in array order (pairs that share a canvas are blended in that order).  Every pair's
 * results are those of emdq_warm_start, emdq_fit_batch_ex, emdq_field (EMDQ_BF16) and
 * mosaic_warp on the same arguments.  Capturable into a CUDA graph.
 *
 *   pairs        host array of `count` descriptors (1..64)
 *   prm          host; NULL = defaults; alpha = 0 derives each pair's from its frame size
 *   warm_params  device, emdq_mlp_param_count() floats, or NULL
 *   fit_ctas     host, count ints (emdq_fit_batch_ex), or NULL
 *   workspace    device, emdq_batch_workspace_size(pairs, count, warm_params != NULL) bytes,
 *                256-byte aligned, not shared with a call in flight
 */
typedef struct {
    const float *src, *dst;         /* device, n x 2 float: the matches */
    int n, frame_w, frame_h;
    const uint8_t *frame;           /* device, frame t: frame_h rows of frame_pitch bytes */
    int channels, frame_pitch;
    int grid_x0, grid_y0, grid_w, grid_h;   /* the window, reference coordinates */
    uint8_t *canvas;                /* device, canvas_h rows of canvas_pitch bytes (4 per pixel) */
    int canvas_w, canvas_h, canvas_pitch, origin_x, origin_y;
    float *q_out, *c_out;           /* device, n x 8 and n float (written) */
    float *p_out;                   /* device, n float (written) or NULL */
    emdq_fit_info *info;            /* device (written) */
} emdq_pair;

EMDQ_API size_t      emdq_batch_workspace_size(const emdq_pair *pairs, int count, int warm);
EMDQ_API emdq_status emdq_batch(const emdq_pair *pairs, int count, const emdq_params *prm,
                                const float *warm_params, const int *fit_ctas, void *workspace,
                                size_t workspace_bytes, void *stream);
/* emdq_batch with the fits in phases (emdq_fit_batch_phases; fit_phases: host, nphases round
 * counts; every pair's p_out non-NULL; not together with fit_ctas, else EMDQ_EINVAL).
 * fit_phases = NULL is emdq_batch. */
EMDQ_API emdq_status emdq_batch_ex(const emdq_pair *pairs, int count, const emdq_params *prm,
                                   const float *warm_params, const int *fit_ctas,
                                   const int *fit_phases, int nphases, void *workspace,
                                   size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ emdq_mosaic ------
 * emdq_field (EMDQ_BF16) and mosaic_warp fused in one tensor-core pass: for every grid
 * pixel the displacement of Eqs. 1-4 is computed exactly as emdq_field computes it and
 * the frame is then blended into the canvas exactly as mosaic_warp blends it, so the
 * canvas ends as the two calls would leave it, without the field going through memory.
 * Arguments: those of emdq_field (q, c, src, n, grid, alpha; workspace of
 * emdq_field_workspace_size(n, grid_w, grid_h, EMDQ_BF16) bytes) and of mosaic_warp
 * (frame, canvas, origin); the same errors.
 */
EMDQ_API emdq_status emdq_mosaic(const float *q, const float *c, const float *src, int n,
                        int grid_x0, int grid_y0, int grid_w, int grid_h, float alpha,
                        const uint8_t *frame, int fw, int fh, int channels, int frame_pitch,
                        uint8_t *canvas, int canvas_w, int canvas_h, int canvas_pitch,
                        int origin_x, int origin_y, void *workspace, size_t workspace_bytes,
                        void *stream);

/* ------------------------------------------------------------------ emdq_mosaic_batch -
 * The dense field and the mosaic update of a group of frames of one sequence in one pass
 * (Eqs. 1-4 and Sec. III-F, Eqs. 23-24, as emdq_field_batch followed by mosaic_warp_batch
 * compute them).  The canvas ends bit for bit as after emdq_field_batch of the problems and
 * mosaic_warp_batch of their frames, in order; the field itself is never written.  One
 * operand-preparation launch, then one persistent tensor-core launch over the tiles of the
 * union of the windows: for each tile the frames whose window meets it, in order, each
 * frame's field of the tile followed at every pixel by the frame's sample at p + d(p) and the
 * capped running average, the canvas words held on chip from the tile's first frame to its
 * last.  Not a step of the paper: a fusion of two of its steps.  emdq_mosaic is this call
 * with one frame.
 *
 *   problems      host array of `count` descriptors (1 <= count <= 16): each frame's fit (q,
 *                 c, src, n as emdq_field), its window (grid_*, reference coordinates; not
 *                 empty; inside the canvas after the origin shift), alpha, and `frame`, the
 *                 device frame t (fw x fh, `channels` 1 or 3, rows `frame_pitch` bytes apart)
 *   canvas        device, 4-byte pixels (c0, c1, c2, w) as mosaic_warp, origin as mosaic_warp;
 *                 no other call may write the union of the windows while this one runs
 *   tile_rows     (_ex) the tiles' pixel rows: 16, 24, 32 or 40 (the default)
 *   workspace     device scratch of emdq_mosaic_batch_workspace_size(problems, count) bytes,
 *                 256-byte aligned, not shared with a call in flight
 * Asynchronous on `stream`.  Returns EMDQ_EINVAL for a bad descriptor or a window outside the
 * canvas, EMDQ_ENOTSUP for count > 16, another tile height, a frame of 2^31 bytes or more or a
 * device without tcgen05, EMDQ_EWORKSPACE / EMDQ_ECUDA as emdq_field; a bounded device wait
 * that gives up (about 2 s) is recorded as EMDQ_ETIMEOUT in the workspace's first word (the
 * canvas is then undefined).
 */
typedef struct {
    const float *q;             /* device, n x 8 warp rows (emdq_fit's q_out) */
    const float *c;             /* device, n field weights (emdq_fit's c_out) */
    const float *src;           /* device, n x 2 match positions in the reference frame */
    int n;
    int grid_x0, grid_y0, grid_w, grid_h;   /* the pixel window, reference coordinates */
    float alpha;                /* Gaussian weight exp(-alpha |p - x_i|^2) */
    const uint8_t *frame;       /* device frame t */
} emdq_mosaic_problem;

EMDQ_API size_t      emdq_mosaic_batch_workspace_size(const emdq_mosaic_problem *problems, int count);
EMDQ_API emdq_status emdq_mosaic_batch(const emdq_mosaic_problem *problems, int count, int fw,
                                       int fh, int channels, int frame_pitch, uint8_t *canvas,
                                       int canvas_w, int canvas_h, int canvas_pitch, int origin_x,
                                       int origin_y, void *workspace, size_t workspace_bytes,
                                       void *stream);
EMDQ_API emdq_status emdq_mosaic_batch_ex(const emdq_mosaic_problem *problems, int count, int fw,
                                          int fh, int channels, int frame_pitch, uint8_t *canvas,
                                          int canvas_w, int canvas_h, int canvas_pitch,
                                          int origin_x, int origin_y, int tile_rows,
                                          void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ emdq_mosaic_pairs -
 * The dense field and the mosaic update of up to 16 independent pairs in one pass (Eqs. 1-4
 * and Sec. III-F, Eqs. 23-24): each pair has its own frame (size and pitch), window and
 * canvas, and each pair's canvas ends bit for bit as after emdq_field (EMDQ_BF16) and
 * mosaic_warp of that pair; the field itself is never written.  One operand-preparation
 * launch, then one persistent tensor-core launch over the tiles of every pair's window (the
 * tiles of emdq_mosaic_batch, 128 x 40 pixels), each tile's field followed at every pixel by
 * the pair's frame sampled at p + d(p) and the capped running average.  Not a step of the
 * paper: the fusion of two of its steps for a batch of unrelated pairs.
 *
 *   pairs         host array of `count` descriptors (1 <= count <= 16): a fit (q, c, src, n
 *                 as emdq_field), its window (grid_*, reference coordinates; not empty;
 *                 inside the pair's canvas after the origin shift), alpha, the device frame
 *                 t (fw x fh, rows frame_pitch bytes apart), and the device canvas (4-byte
 *                 pixels (c0, c1, c2, w) as mosaic_warp; canvas_pitch bytes per row) with the
 *                 origin of the reference frame in it
 *   channels      1 or 3, the same for every pair
 *   workspace     device scratch of emdq_mosaic_pairs_workspace_size(pairs, count) bytes,
 *                 256-byte aligned, not shared with a call in flight
 * The pairs' tiles run in no fixed order, so no two pairs may update the same canvas bytes:
 * EMDQ_EINVAL if the spans of canvas rows of two pairs' windows (first to last byte)
 * overlap.  Asynchronous on `stream`.  Returns EMDQ_EINVAL for a bad descriptor or a window
 * outside its canvas, EMDQ_ENOTSUP for count > 16, a frame of 2^31 bytes or more or a device
 * without tcgen05, EMDQ_EWORKSPACE / EMDQ_ECUDA as emdq_field; a bounded device wait that
 * gives up (about 2 s) is recorded as EMDQ_ETIMEOUT in the workspace's first word (the
 * canvases are then undefined).
 */
typedef struct {
    const float *q;             /* device, n x 8 warp rows (emdq_fit's q_out) */
    const float *c;             /* device, n field weights (emdq_fit's c_out) */
    const float *src;           /* device, n x 2 match positions in the reference frame */
    int n;
    int grid_x0, grid_y0, grid_w, grid_h;   /* the pixel window, reference coordinates */
    float alpha;                /* Gaussian weight exp(-alpha |p - x_i|^2) */
    const uint8_t *frame;       /* device frame t: fh rows of frame_pitch bytes */
    int fw, fh, frame_pitch;
    uint8_t *canvas;            /* device, canvas_h rows of canvas_pitch bytes */
    int canvas_w, canvas_h, canvas_pitch, origin_x, origin_y;
} emdq_mosaic_pair;

EMDQ_API size_t      emdq_mosaic_pairs_workspace_size(const emdq_mosaic_pair *pairs, int count);
EMDQ_API emdq_status emdq_mosaic_pairs(const emdq_mosaic_pair *pairs, int count, int channels,
                                       void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ learned warm start
 * Not in the paper (the paper's EMDQ starts EM without a prior).  A 16-64-64-1 network
 * predicts each match's initial inlier weight p0 for emdq_fit from its 8 nearest
 * matches, so that EM starts closer to its answer and needs fewer iterations; plain EM
 * (p0 = NULL) remains the fallback.  Inference and training run in these kernels.
 *
 * Features of match j (feat_out row, 16 floats), k over the 8 nearest matches by
 * |x_k - x_j| (float32 squared distances, ties to the lower index), in pixels:
 *   log(1 + |(y_k - x_k) - (y_j - x_j)|) for the 8 k, sorted ascending (k's residual
 *     under the translation j implies: no fit needed, robust to many outliers), then
 *   log(1 + |x_k - x_j|) for the 8 k, ascending (the scale for judging those residuals).
 * Network parameters (emdq_mlp_param_count() = 5313 floats, device): W1[64][16], b1[64],
 * W2[64][64], b2[64], W3[64], b3; ReLU hidden layers, logistic output.  The forward rounds
 * parameters, inputs and hidden activations to BF16 and accumulates in FP32.
 *
 * emdq_mlp_train_step: mean binary cross-entropy over `batch` samples (feat rows, labels
 * 0/1); writes the mean gradient to grad_out and the mean loss to loss_out (each may be
 * NULL); if step >= 1, applies Adam step number `step` (beta1 0.9, beta2 0.999,
 * eps 1e-8, learning rate lr) to the FP32 params with moments adam_m, adam_v (5313 floats
 * each, zero before step 1).  step = 0 computes the gradient only.
 */
EMDQ_API int         emdq_mlp_param_count(void);
EMDQ_API emdq_status emdq_warm_features(const float *src, const float *dst, int n,
                                        float *feat_out, void *stream);
EMDQ_API emdq_status emdq_warm_infer(const float *feat, int n, const float *params,
                                     float *p0_out, void *stream);
/* Features and network for `count` problems (1..64) in one launch: host arrays of device
 * pointers src[b], dst[b] (n[b] x 2 float) and p0_out[b] (n[b] float, written); the same
 * p0 as emdq_warm_features followed by emdq_warm_infer. */
EMDQ_API emdq_status emdq_warm_start(const float *const *src, const float *const *dst,
                                     const int *n, float *const *p0_out, int count,
                                     const float *params, void *stream);
EMDQ_API size_t      emdq_mlp_train_workspace_size(int batch);
EMDQ_API emdq_status emdq_mlp_train_step(const float *feat, const float *label, int batch,
                                         float *params, float *adam_m, float *adam_v,
                                         int step, float lr, float *grad_out, float *loss_out,
                                         void *workspace, size_t workspace_bytes,
                                         void *stream);

/* Sec. III-F: "frame 0 is inserted directly" -- copy the reference frame into the canvas
 * at the origin with merge weight 1. */
EMDQ_API emdq_status mosaic_insert_reference(const uint8_t *frame, int fw, int fh, int channels,
                                    int frame_pitch, uint8_t *canvas, int canvas_w,
                                    int canvas_h, int canvas_pitch, int origin_x,
                                    int origin_y, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* EMDQ_H */
