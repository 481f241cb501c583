// Dense field on the 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulate).
//
// The Gaussian of Eq. 4 separates on a pixel grid,
//     exp(-alpha |p - x_i|^2) = exp(-alpha (p_x - x_i)^2) exp(-alpha (p_y - y_i)^2),
// so the six blend sums of Eqs. 2-3 (four DQ components and the scale, each relative to a
// reference row, and the weight) are, per channel ch, a GEMM over the matches:
//     F_ch[p_x, p_y] = sum_i Ex[p_x, i] * G_ch[p_y, i],
//     Ex[p_x, i] = exp(-alpha (p_x - x_i)^2),
//     G_ch[p_y, i] = c_i exp(-alpha (p_y - y_i)^2) (Q_i,ch - Q_ref,ch)   (ch < 5),
//     G_5[p_y, i]  = c_i exp(-alpha (p_y - y_i)^2).
// This is the same sum as the per-pixel definition, with (w + h) N exponentials instead
// of w h N.  Subtracting the reference row (exact: the blend is linear) keeps the BF16
// rounding of G off the large scale and dual-part values the pixel position multiplies.
//
// field_tc_prep_kernel writes Ex (K-major rows of pixels x) and G (K-major rows of
// pixels y, six channel planes) as BF16 into the workspace, zero-padded to whole tiles.
// Its K columns are only the matches of nonzero weight c_i (the EM outliers have c = 0
// and add exactly nothing), so the GEMM's K shrinks by the outlier fraction; the column
// count goes to the GEMM through device memory.
// field_tc_kernel: persistent, one CTA per SM looping over 128 x 32 pixel tiles, warp
// specialised.  Warp 0 (one thread) streams 64-match slices of Ex (128 rows) and of G
// (6 x 32 rows, one 3-D box) through a 4-stage shared-memory ring with TMA; warp 1 (one
// thread) issues tcgen05.mma (M = 128 pixels x, N = 192 = 6 channels x 32 pixels y,
// K = 16) into one of two TMEM accumulators; the epilogue warps read the other
// accumulator back with tcgen05.ld (thread = pixel x = TMEM lane; for the field two warps
// per lane quadrant, each taking half of the 32 pixel rows) and evaluate Eq. 1, so the
// epilogue of a tile overlaps the MMAs of the next.
// mosaic_tc_kernel: the same GEMM over the tiles of the union of a group of frames' windows,
// each tile taken through the frames whose window meets it, in order; its epilogue goes on
// from each pixel's displacement to the frame's sample and the canvas update (the
// stand-alone warp's per-pixel code), with the tile's canvas words held in registers from
// its first frame to its last, so the field never visits HBM.
#include <cmath>
#include <mutex>
#include <vector>

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "blend.cuh"
#include "field.cuh"
#include "field_tc.cuh"
#include "tc_ptx.cuh"

namespace emdq {

constexpr int kTcM = 128;                // pixels x per tile (MMA M, TMEM lanes)
constexpr int kTcCh = 6;                 // dr_w, dr_z, dd_x, dd_y, ds, weight
constexpr int kTcK = 64;                 // matches per stage: one 128-byte swizzle row
constexpr int kTcStages = 4;
// Pixel rows per tile (PY): MMA N = 6 PY.  32 is the default; the autotuner may choose
// another per size class (more rows: more MACs per operand byte and per MMA; fewer rows:
// more tiles, for windows too small to fill every SM).
constexpr int kTcPYDefault = 32;
constexpr int kTcPYChoices[4] = {16, 24, 32, 40};
constexpr int kTcPYMax = 40;
// Epilogue warps: two per TMEM lane quadrant for the field (each half of the pixel rows);
// five per quadrant for the fused field + warp, whose epilogue issues ~200 instructions and
// two dependent memory round trips per pixel and frame (one warp per 8-row group of a
// 40-row tile: with fewer, the epilogue, not the MMA, sets the rate).  Threads: producer
// warp, MMA warp, epilogue warps.
constexpr int kTcEpiWarps = 8;
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;
constexpr int kMosEpiWarps = 20;
constexpr int kMosThreads = 64 + 32 * kMosEpiWarps;
constexpr int kMosPYDefault = 40;
constexpr uint32_t kTcABytes = kTcM * kTcK * 2;
constexpr uint32_t kTcAccCols = 256;     // one accumulator: 6 PY <= 240 columns used
constexpr uint32_t kTcTmemCols = 2 * kTcAccCols;

template <int PY>
struct TcShape {
    static constexpr int N = kTcCh * PY;                       // MMA N
    static constexpr uint32_t BBytes = N * kTcK * 2;
    static constexpr uint32_t StageBytes = kTcABytes + BBytes;
    static constexpr size_t SmemBytes = kTcStages * StageBytes + 1024 /*barriers*/ + 1024 /*align*/;
    static constexpr uint32_t Idesc = tc::idesc_bf16_f32(kTcM, N);
    static_assert(PY % 8 == 0 && N % 16 == 0 && N <= 240, "MMA N for M = 128 (one accumulator)");
    static_assert(StageBytes % 1024 == 0 && kTcABytes % 1024 == 0, "SW128 tiles 1 KiB aligned");
    static_assert((PY * 128) % 1024 == 0 || PY % 8 == 0, "8-row groups of the B planes");
};
constexpr size_t kTcSmemMax = TcShape<kTcPYMax>::SmemBytes;
// Operand rows per prep block: each block pays one chain of dependent loads (the
// nonzero-weight columns, the reference row, its columns' data) before writing rows, so
// blocks take many rows; G rows carry six planes, so they take fewer than Ex rows.
constexpr int kPrepRowsA = 32;
constexpr int kPrepRowsB = 16;
constexpr int kPrepThreads = 256;
constexpr long long kWaitLimit = 4000000000LL;   // SM cycles (about 2 s)

struct TcGeom {
    int kp;          // matches padded to kTcK
    int wp, hp;      // grid padded to kTcM, the tile's PY rows
    size_t a_bytes, b_bytes;
};

__host__ __device__ inline TcGeom tc_geom(int n, int gw, int gh, int py)
{
    TcGeom g;
    g.kp = (n + kTcK - 1) / kTcK * kTcK;
    g.wp = (gw + kTcM - 1) / kTcM * kTcM;
    g.hp = (gh + py - 1) / py * py;
    g.a_bytes = (size_t)g.wp * g.kp * 2;
    g.b_bytes = (size_t)kTcCh * g.hp * g.kp * 2;
    return g;
}

// Operand bytes of a problem for whichever tile height is chosen (the largest padding).
inline size_t tc_operand_bytes_max(int n, int gw, int gh)
{
    size_t b = 0;
    for (int py : kTcPYChoices) {
        const TcGeom g = tc_geom(n, gw, gh, py);
        const size_t v = ((g.a_bytes + 1023) / 1024 + (g.b_bytes + 1023) / 1024) * 1024;
        b = v > b ? v : b;
    }
    return b;
}

// The displacement d = W(p) - p of pixel p from its six accumulated sums (Eqs. 1-3): the
// blended row is the reference row plus the weighted differences over their weight w > 0,
// then the blend is normalised and applied.  Both reciprocals (1/w and the real part's
// 1/|r|^2) are the single-instruction approximation (rcp.approx.ftz: within one ulp), not
// the correctly rounded division: an error of 2^-23 relative in a displacement of a few
// thousand pixels is far below the BF16 operands' 2^-9, and the division sequences were
// about a tenth of the fused epilogue's instructions.  The field call and the fused field +
// warp call both take d from here, so their canvases stay the same bits.
__device__ __forceinline__ float2 tc_displacement(float f0, float f1, float f2, float f3, float f4,
                                                  float w, float ra, float rb, float ru, float rv,
                                                  float rs, float px, float py)
{
    const float inv = rcp_approx_ftz(w);
    const float a = ra + f0 * inv, b = rb + f1 * inv, u = ru + f2 * inv, v = rv + f3 * inv;
    const float s = rs + f4 * inv;
    const float in2 = rcp_approx_ftz(a * a + b * b);
    const float ct = (a * a - b * b) * in2;
    const float st = 2.0f * a * b * in2;
    const float tx = 2.0f * (a * u - b * v) * in2;
    const float ty = 2.0f * (b * u + a * v) * in2;
    return make_float2(s * (ct * px - st * py + tx) - px, s * (st * px + ct * py + ty) - py);
}

// Columns of the GEMM: the matches with c_i != 0 in index order (a match of weight 0 adds
// exactly nothing to any of the six sums), found by every block with the same block scan.
// Returns their number m; col(k) = the k-th such match.  Above kCompactMax matches the
// columns are all matches, in order.
constexpr int kCompactMax = 8192;

__device__ int compact_columns(const float *__restrict__ c, int n, int *s_idx)
{
    __shared__ int s_warp[kPrepThreads / 32];
    if (n > kCompactMax) return -1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // thread t owns matches [t per, (t + 1) per): one flag bit each (per <= 32); all its
    // loads are issued before any is used (one memory round trip)
    const int per = (n + kPrepThreads - 1) / kPrepThreads;
    const int k0 = threadIdx.x * per;
    float cv[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        const int k = k0 + u;
        cv[u] = (u < per && k < n) ? c[k] : 0.f;
    }
    unsigned mask = 0;
#pragma unroll
    for (int u = 0; u < 32; ++u)
        if (cv[u] != 0.f) mask |= 1u << u;
    const int cnt = __popc(mask);
    int incl = cnt;                                   // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int off = incl - cnt, tot = 0;
#pragma unroll
    for (int w = 0; w < kPrepThreads / 32; ++w) {
        const int cw = s_warp[w];
        off += w < warp ? cw : 0;
        tot += cw;
    }
    for (; mask; mask &= mask - 1) s_idx[off++] = k0 + __ffs(mask) - 1;
    __syncthreads();
    return tot;
}

// A batch of fields (frames or pairs) run by one prep launch and one GEMM launch, so the
// fixed costs of the two launches are paid once per batch.
constexpr int kFieldBatchMax = 16;

struct TcProblem {
    const float *q, *c;
    const float2 *src;
    int n, kp, gx0, gy0, gw, gh, wp, hp;
    float alpha;
    __nv_bfloat162 *A, *B;       // BF16 operands (workspace)
    float *ref;                  // reference row, 6 floats (workspace or caller)
    int *kcount;                 // K columns the prep wrote (workspace)
    float2 *disp;                // the displacement field (field_tc_kernel)
    int ntx, tile0, ntiles;      // GEMM tiles [tile0, tile0 + ntiles) of the batch
    int block0, a_blocks, nblocks;   // prep blocks [block0, block0 + nblocks), Ex rows first
};

struct TcBatch {
    CUtensorMap tmA[kFieldBatchMax];
    CUtensorMap tmB[kFieldBatchMax];
    TcProblem p[kFieldBatchMax];
    int count, total_tiles;
    int *err;                    // device status (ETIMEOUT), cleared by the prep launch
};

__device__ __forceinline__ int problem_of_block(const TcBatch &Bt, int blk)
{
    int b = 0;
    while (b + 1 < Bt.count && Bt.p[b + 1].block0 <= blk) ++b;
    return b;
}

__device__ __forceinline__ int problem_of_tile(const TcBatch &Bt, int tile)
{
    int b = 0;
    while (b + 1 < Bt.count && Bt.p[b + 1].tile0 <= tile) ++b;
    return b;
}

__global__ void __launch_bounds__(kPrepThreads) field_tc_prep_kernel(const __grid_constant__ TcBatch Bt)
{
    __shared__ int s_idx[kCompactMax];
    const TcProblem &P = Bt.p[problem_of_block(Bt, blockIdx.x)];
    const int blk = blockIdx.x - P.block0;
    const float *__restrict__ q = P.q;
    const float *__restrict__ c = P.c;
    const float2 *__restrict__ src = P.src;
    const int n = P.n, wp = P.wp, hp = P.hp, gw = P.gw, gh = P.gh;
    // exp(-alpha d^2) = 2^(-alpha log2(e) d^2) with MUFU.EX2 (the BF16 rounding of the
    // operands dominates its error)
    const float alpha2 = P.alpha * 1.4426950408889634f;
    const int half = P.kp / 2;
    const int mc = compact_columns(c, n, s_idx);
    const bool compact = mc >= 0;
    const int m = compact ? mc : n;
    // columns written: m rounded up to whole 64-match slices (at least one), zeros past m
    const int kc = m > 0 ? (m + kTcK - 1) / kTcK * kTcK : kTcK;
    const int halfc = kc / 2;
    if (blk == 0 && threadIdx.x == 0) *P.kcount = kc;
    if (blockIdx.x == 0 && threadIdx.x == 0) *Bt.err = 0;   // raised by the GEMM only after its wait
    auto col = [&](int k) { return compact ? s_idx[k] : k; };
    if (blk < P.a_blocks) {
        __nv_bfloat162 *__restrict__ A = P.A;
        const int r0 = blk * kPrepRowsA;
        for (int k2 = threadIdx.x; k2 < halfc; k2 += kPrepThreads) {
            const int k0 = 2 * k2, k1 = k0 + 1;
            const float x0 = k0 < m ? src[col(k0)].x : 0.f, x1 = k1 < m ? src[col(k1)].x : 0.f;
            for (int r = 0; r < kPrepRowsA; ++r) {
                const int px = r0 + r;
                if (px >= wp) break;
                const float p = static_cast<float>(P.gx0 + px);
                const bool row = px < gw;
                const float d0 = p - x0, d1 = p - x1;
                const float e0 = (row && k0 < m) ? ex2_ftz(-alpha2 * d0 * d0) : 0.f;
                const float e1 = (row && k1 < m) ? ex2_ftz(-alpha2 * d1 * d1) : 0.f;
                A[(size_t)px * half + k2] = __floats2bfloat162_rn(e0, e1);
            }
        }
    } else {
        __nv_bfloat162 *__restrict__ B = P.B;
        const int r0 = (blk - P.a_blocks) * kPrepRowsB;
        __shared__ float red[6 * 32];
        float rf[6];
        reference_row(q, c, n, red, rf);      // same bits in every block
        if (blk == P.a_blocks && threadIdx.x == 0)
            for (int k = 0; k < 6; ++k) P.ref[k] = rf[k];
        for (int k2 = threadIdx.x; k2 < halfc; k2 += kPrepThreads) {
            const int k0 = 2 * k2;
            float y[2] = {0.f, 0.f}, cw[2] = {0.f, 0.f}, cq[2][5];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int kk = k0 + u;
#pragma unroll
                for (int ch = 0; ch < 5; ++ch) cq[u][ch] = 0.f;
                if (kk < m) {
                    const int k = col(kk);
                    y[u] = src[k].y;
                    cw[u] = c[k];
                    const float4 r = *reinterpret_cast<const float4 *>(q + 8 * (size_t)k);
                    const float s = q[8 * (size_t)k + 4];
                    cq[u][0] = cw[u] * (r.x - rf[0]);
                    cq[u][1] = cw[u] * (r.y - rf[1]);
                    cq[u][2] = cw[u] * (r.z - rf[2]);
                    cq[u][3] = cw[u] * (r.w - rf[3]);
                    cq[u][4] = cw[u] * (s - rf[4]);
                }
            }
            for (int r = 0; r < kPrepRowsB; ++r) {
                const int py = r0 + r;
                if (py >= hp) break;
                const float p = static_cast<float>(P.gy0 + py);
                const bool row = py < gh;
                const float d0 = p - y[0], d1 = p - y[1];
                const float e0 = row ? ex2_ftz(-alpha2 * d0 * d0) : 0.f;
                const float e1 = row ? ex2_ftz(-alpha2 * d1 * d1) : 0.f;
#pragma unroll
                for (int ch = 0; ch < 5; ++ch)
                    B[((size_t)ch * hp + py) * half + k2] =
                        __floats2bfloat162_rn(e0 * cq[0][ch], e1 * cq[1][ch]);
                B[((size_t)5 * hp + py) * half + k2] = __floats2bfloat162_rn(e0 * cw[0], e1 * cw[1]);
            }
        }
    }
    // this block's rows are written: the GEMM launched after this kernel may start its
    // set-up once every block is here (it still waits, griddepcontrol.wait, for the whole
    // grid before it reads the operands).  Triggered only now, so that the GEMM's large
    // CTAs do not crowd the prep blocks out of the SMs.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The displacement field of every problem of the batch, tiles of kTcM x PY pixels.
template <int PY>
__global__ void __launch_bounds__(kTcThreads, 1) field_tc_kernel(const __grid_constant__ TcBatch Bt)
{
    using S = TcShape<PY>;
    constexpr uint32_t kTcStageBytes = S::StageBytes;
    constexpr uint32_t kTcIdesc = S::Idesc;
    const int ntiles = Bt.total_tiles;
    int *__restrict__ err = Bt.err;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kTcStages * kTcStageBytes);
    uint64_t *empty = full + kTcStages;
    uint64_t *acc_full = empty + kTcStages;     // [2] MMA -> epilogue
    uint64_t *acc_empty = acc_full + 2;         // [2] epilogue -> MMA (every epilogue warp arrives)
    uint64_t *done = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int *issued = const_cast<int *>(abort_flag + 1);     // chunks whose loads were issued
    int *consumed = issued + 1;                          // chunks whose MMAs were issued
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            tc::mbar_init(full + s, 1);
            tc::mbar_init(empty + s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(acc_full + a, 1);
            tc::mbar_init(acc_empty + a, kTcEpiWarps);
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
        *issued = 0;
        *consumed = 0;
        tc::fence_mbar_init();
        for (int b = 0; b < Bt.count; ++b) {
            tc::prefetch_tmap(&Bt.tmA[b]);
            tc::prefetch_tmap(&Bt.tmB[b]);
        }
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, kTcTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    // everything above is independent of the prep kernel (programmatic dependent launch);
    // its operands, column count and reference row are read only after this wait
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer: every tile of this CTA, every 64-match slice
            int chunk = 0;
            for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
                const int b = problem_of_tile(Bt, tile);
                const TcProblem &P = Bt.p[b];
                const int lt = tile - P.tile0, tx = lt % P.ntx, ty = lt / P.ntx;
                // 64-match slices along K: the prep kernel's column count (the matches of
                // nonzero weight), a whole number of slices, at least one
                const int nchunks = *P.kcount / kTcK;
                for (int k = 0; k < nchunks; ++k, ++chunk) {
                    const int s = chunk % kTcStages;
                    const uint32_t ph = (chunk / kTcStages) & 1;
                    if (chunk >= kTcStages && !tc::mbar_wait(empty + s, ph ^ 1, kWaitLimit, false)) {
                        *abort_flag = 1;
                        break;
                    }
                    uint8_t *sa = smem + s * kTcStageBytes;
                    tc::mbar_arrive_expect_tx(full + s, kTcStageBytes);
                    tc::tma_load_2d(sa, &Bt.tmA[b], full + s, k * kTcK, tx * kTcM);
                    tc::tma_load_3d(sa + kTcABytes, &Bt.tmB[b], full + s, k * kTcK, ty * PY, 0);
                    *issued = chunk + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: accumulator it & 1 of tile iteration it
            int chunk = 0, it = 0;
            for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++it) {
                const int a = it & 1;
                if (it >= 2 && !tc::mbar_wait(acc_empty + a, ((it >> 1) - 1) & 1, kWaitLimit, false)) {
                    *abort_flag = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d = tmem + a * kTcAccCols;
                const int nchunks = *Bt.p[problem_of_tile(Bt, tile)].kcount / kTcK;
                bool ok = true;
                for (int k = 0; k < nchunks; ++k, ++chunk) {
                    const int s = chunk % kTcStages;
                    const uint32_t ph = (chunk / kTcStages) & 1;
                    if (!tc::mbar_wait(full + s, ph, kWaitLimit, false)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t sa = tc::smem_u32(smem + s * kTcStageBytes);
                    const uint32_t sb = sa + kTcABytes;
#pragma unroll
                    for (int kk = 0; kk < kTcK / 16; ++kk) {
                        // advance 16 BF16 = 32 bytes along K inside the 128-byte swizzled row
                        tc::mma_f16(d, tc::desc_kmajor_sw128(sa + kk * 32),
                                    tc::desc_kmajor_sw128(sb + kk * 32), kTcIdesc, (k | kk) != 0);
                    }
                    tc::mma_commit(empty + s);
                    *consumed = chunk + 1;
                }
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                tc::mma_commit(acc_full + a);
            }
            tc::mma_commit(done);   // tracks every MMA issued above, also after an abort
        }
    } else {
        // epilogue warps: TMEM lane quadrant q = warp % 4 (the lanes a warp may access),
        // thread = pixel x of the tile; the tile's groups of 8 pixel rows are dealt to the
        // warp sets in turn (with 8 warps: warps 2-5 take groups 0, 2, ..., warps 6-9 groups
        // 1, 3, ...)
        constexpr int kSets = kTcEpiWarps / 4;
        constexpr int kAllGroups = PY / 8;
        const int q = warp & 3;
        const int g0 = (warp - 2) >> 2;
        const int g_last = g0 + (kAllGroups - 1 - g0) / kSets * kSets;
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int a = it & 1;
            const bool ok = tc::mbar_wait(acc_full + a, (it >> 1) & 1, kWaitLimit, true);
            tc::fence_after_sync();
            if (!ok || *abort_flag) {
                *abort_flag = 1;
                break;
            }
            const TcProblem &P = Bt.p[problem_of_tile(Bt, tile)];
            const int gx0 = P.gx0, gy0 = P.gy0, gw = P.gw, gh = P.gh;
            float2 *__restrict__ disp = P.disp;
            const float ra = P.ref[0], rb = P.ref[1], ru = P.ref[2], rv = P.ref[3], rs = P.ref[4];
            const int lt = tile - P.tile0, tx = lt % P.ntx, ty = lt / P.ntx;
            const int x = tx * kTcM + q * 32 + lane;
            const float px = static_cast<float>(gx0 + x);
            const uint32_t lane_base = tmem + a * kTcAccCols + (static_cast<uint32_t>(q * 32) << 16);
#pragma unroll 1
            for (int g = g0; g < kAllGroups; g += kSets) {
                float F[kTcCh][8];
#pragma unroll
                for (int ch = 0; ch < kTcCh; ++ch) tc::tmem_ld_x8(lane_base + ch * PY + g * 8, F[ch]);
                tc::tmem_wait_ld();
                if (g == g_last) {
                    // the accumulator has been read: hand it back to the MMA warp
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(acc_empty + a);
                }
                float2 d[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float py = static_cast<float>(gy0 + ty * PY + g * 8 + j);
                    d[j] = make_float2(NAN, NAN);
                    if (F[5][j] > 0.f)
                        d[j] = tc_displacement(F[0][j], F[1][j], F[2][j], F[3][j], F[4][j], F[5][j],
                                               ra, rb, ru, rv, rs, px, py);
                }
                const int y0 = ty * PY + g * 8;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (x < gw && y0 + j < gh) disp[(size_t)(y0 + j) * gw + x] = d[j];
            }
        }
    }
    __syncwarp();
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        // every MMA issued has completed before the accumulators are released
        tc::mbar_wait(done, 0, kWaitLimit, true);
        if (*abort_flag) {
            atomicMax(err, (int)EMDQ_ETIMEOUT);
            // drain loads that were issued but never consumed before the CTA exits
            for (int k = *consumed; k < *issued; ++k)
                tc::mbar_wait(full + (k % kTcStages), (k / kTcStages) & 1, kWaitLimit, true);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, kTcTmemCols);
}

// ------------------------------------------------------------------------- fused mosaic
// A pair's own canvas and frame geometry (independent pairs, emdq_mosaic_pairs).
struct MosaicTarget {
    uchar4 *canvas;
    int cpitch4, ox, oy;
    int fw, fh, pitch;
};

// Frames and canvas of a group of frames blended in one pass; the tiles are those of the
// union of the group's windows (reference coordinates).  For independent pairs (PAIRS
// kernels) every problem has its own canvas and frame geometry in tgt[] and the tiles are
// those of each problem's own window (the GEMM's tiles: Bt.p[b].tile0 ...).
struct MosaicBatch {
    const uint8_t *frame[kFieldBatchMax];
    int fw, fh, pitch;
    uchar4 *canvas;
    int cpitch4, ox, oy;
    int ux0, uy0, uw, uh;     // union of the windows
    int ntx, ntiles;          // tiles across / in all of the union (PAIRS: all problems' tiles)
    MosaicTarget tgt[kFieldBatchMax];
};

// Does problem P's window meet the tile at (x0, y0)?
template <int PY>
__device__ __forceinline__ bool tile_meets(const TcProblem &P, int x0, int y0)
{
    return x0 < P.gx0 + P.gw && x0 + kTcM > P.gx0 && y0 < P.gy0 + P.gh && y0 + PY > P.gy0;
}

// The first problem after b whose window meets the tile (Bt.count if none).
template <int PY>
__device__ __forceinline__ int next_meeting(const TcBatch &Bt, int b, int x0, int y0)
{
    for (++b; b < Bt.count; ++b)
        if (tile_meets<PY>(Bt.p[b], x0, y0)) break;
    return b;
}

// A tile's origin and its first item (Bt.count: none): the union's tiles and the frames
// meeting each, or (PAIRS) each problem's own tiles, one item each.
template <int PY, bool PAIRS>
__device__ __forceinline__ int tile_first(const TcBatch &Bt, const MosaicBatch &M, int tile, int &x0,
                                          int &y0)
{
    if (PAIRS) {
        const int b = problem_of_tile(Bt, tile);
        const TcProblem &P = Bt.p[b];
        const int l = tile - P.tile0;
        x0 = P.gx0 + (l % P.ntx) * kTcM;
        y0 = P.gy0 + (l / P.ntx) * PY;
        return b;
    }
    x0 = M.ux0 + (tile % M.ntx) * kTcM;
    y0 = M.uy0 + (tile / M.ntx) * PY;
    return next_meeting<PY>(Bt, -1, x0, y0);
}

template <int PY, bool PAIRS>
__device__ __forceinline__ int tile_next(const TcBatch &Bt, int b, int x0, int y0)
{
    return PAIRS ? Bt.count : next_meeting<PY>(Bt, b, x0, y0);
}

// The tile of round r for this CTA.  The rounds alternate direction (CTA c takes tile r G + c
// in even rounds, r G + G - 1 - c in odd ones), so that the CTAs that get a tile in a partial
// last round are those that got the last tiles of the round before -- the tiles of a window's
// ragged last rows, whose epilogue is short -- and not those that got full tiles twice.
__device__ __forceinline__ int round_tile(int r)
{
    return r * (int)gridDim.x + ((r & 1) ? (int)gridDim.x - 1 - (int)blockIdx.x : (int)blockIdx.x);
}

// Items: (tile, frame) pairs, tiles of the union in this CTA's turn, the frames meeting each
// in order (PAIRS: a problem's tile and its own frame).  The TMA and MMA warps run them as field_tc_kernel runs tiles (the operand rows
// of the tile's pixels in that frame's operands; outside its padded window TMA fills zeros,
// and outside its window the operands are zero, so the weight channel there is 0).  The
// epilogue warps: TMEM lane quadrant q = warp % 4, thread = pixel x; warp set s (four warps,
// one per quadrant) takes the tile's 8-row groups s, s + kSets, ...; it reads its canvas
// words once per tile, updates them through the tile's frames in order (each pixel's
// displacement from Eq. 1, then the sample and the capped running average of
// mosaic_warp_batch) and writes them back once.
template <int CH, int PY, bool PAIRS>
__global__ void __launch_bounds__(kMosThreads, 1) mosaic_tc_kernel(const __grid_constant__ TcBatch Bt,
                                                                 const __grid_constant__ MosaicBatch M)
{
    using S = TcShape<PY>;
    constexpr uint32_t kStageBytes = S::StageBytes;
    constexpr int kSets = kMosEpiWarps / 4;
    constexpr int kAllGroups = PY / 8;
    constexpr int kMyGroups = (kAllGroups + kSets - 1) / kSets;
    int *__restrict__ err = Bt.err;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kTcStages * kStageBytes);
    uint64_t *empty = full + kTcStages;
    uint64_t *acc_full = empty + kTcStages;
    uint64_t *acc_empty = acc_full + 2;
    uint64_t *done = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int *issued = const_cast<int *>(abort_flag + 1);
    int *consumed = issued + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // RN(1 / (w + 1)) for every canvas weight byte w (the blend's divisor; the blend keeps w <= 30,
    // the table covers any byte), one shared load per pixel instead of a reciprocal sequence
    __shared__ float rw1_of[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) rw1_of[i] = __frcp_rn(static_cast<float>(i) + 1.f);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            tc::mbar_init(full + s, 1);
            tc::mbar_init(empty + s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(acc_full + a, 1);
            tc::mbar_init(acc_empty + a, kMosEpiWarps);
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
        *issued = 0;
        *consumed = 0;
        tc::fence_mbar_init();
        for (int b = 0; b < Bt.count; ++b) {
            tc::prefetch_tmap(&Bt.tmA[b]);
            tc::prefetch_tmap(&Bt.tmB[b]);
        }
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, kTcTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    // the prep launch's operands are complete from here on
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp == 0) {
        if (lane == 0) {
            int chunk = 0;
            for (int r = 0, tile = round_tile(0); tile < M.ntiles && !*abort_flag; tile = round_tile(++r)) {
                int x0, y0;
                for (int b = tile_first<PY, PAIRS>(Bt, M, tile, x0, y0); b < Bt.count && !*abort_flag;
                     b = tile_next<PY, PAIRS>(Bt, b, x0, y0)) {
                    const TcProblem &P = Bt.p[b];
                    const int nchunks = *P.kcount / kTcK;
                    for (int k = 0; k < nchunks; ++k, ++chunk) {
                        const int s = chunk % kTcStages;
                        const uint32_t ph = (chunk / kTcStages) & 1;
                        if (chunk >= kTcStages && !tc::mbar_wait(empty + s, ph ^ 1, kWaitLimit, false)) {
                            *abort_flag = 1;
                            break;
                        }
                        uint8_t *sa = smem + s * kStageBytes;
                        tc::mbar_arrive_expect_tx(full + s, kStageBytes);
                        tc::tma_load_2d(sa, &Bt.tmA[b], full + s, k * kTcK, x0 - P.gx0);
                        tc::tma_load_3d(sa + kTcABytes, &Bt.tmB[b], full + s, k * kTcK, y0 - P.gy0, 0);
                        *issued = chunk + 1;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // item it into accumulator it & 1
            int chunk = 0, it = 0;
            bool ok = true;
            for (int r = 0, tile = round_tile(0); tile < M.ntiles && ok; tile = round_tile(++r)) {
                int x0, y0;
                for (int b = tile_first<PY, PAIRS>(Bt, M, tile, x0, y0); b < Bt.count && ok;
                     b = tile_next<PY, PAIRS>(Bt, b, x0, y0), ++it) {
                    const int a = it & 1;
                    if (it >= 2 && !tc::mbar_wait(acc_empty + a, ((it >> 1) - 1) & 1, kWaitLimit, false)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t d = tmem + a * kTcAccCols;
                    const int nchunks = *Bt.p[b].kcount / kTcK;
                    for (int k = 0; k < nchunks; ++k, ++chunk) {
                        const int s = chunk % kTcStages;
                        const uint32_t ph = (chunk / kTcStages) & 1;
                        if (!tc::mbar_wait(full + s, ph, kWaitLimit, false)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t sa = tc::smem_u32(smem + s * kStageBytes);
                        const uint32_t sb = sa + kTcABytes;
#pragma unroll
                        for (int kk = 0; kk < kTcK / 16; ++kk)
                            tc::mma_f16(d, tc::desc_kmajor_sw128(sa + kk * 32),
                                        tc::desc_kmajor_sw128(sb + kk * 32), S::Idesc, (k | kk) != 0);
                        tc::mma_commit(empty + s);
                        *consumed = chunk + 1;
                    }
                    if (ok) tc::mma_commit(acc_full + a);
                }
            }
            if (!ok) *abort_flag = 1;
            tc::mma_commit(done);   // tracks every MMA issued above, also after an abort
        }
    } else {
        const int q = warp & 3;
        const int set = (warp - 2) >> 2;
        const bool idle = set >= kAllGroups;           // no 8-row group for this set
        const int g_last = idle ? 0 : set + (kAllGroups - 1 - set) / kSets * kSets;
        int it = 0;
        bool alive = true;
        for (int r = 0, tile = round_tile(0); tile < M.ntiles && alive; tile = round_tile(++r)) {
            int x0, y0;
            int b = tile_first<PY, PAIRS>(Bt, M, tile, x0, y0);
            if (b >= Bt.count) continue;                 // no window meets this tile
            // the tile's canvas and the end of the pixels it may update: the group's canvas and
            // the union of the windows, or (PAIRS) the pair's canvas and its window
            const int bt = b;
#define EMDQ_TGT(f) (PAIRS ? M.tgt[bt].f : M.f)
#define EMDQ_YE (PAIRS ? Bt.p[bt].gy0 + Bt.p[bt].gh : M.uy0 + M.uh)
            const int x = x0 + q * 32 + lane;
            const bool col_in = x < (PAIRS ? Bt.p[bt].gx0 + Bt.p[bt].gw : M.ux0 + M.uw);
            const float px = static_cast<float>(x);
            uchar4 cv[kMyGroups][8];
#pragma unroll
            for (int gi = 0; gi < kMyGroups; ++gi) {
                const int g = set + gi * kSets;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int y = y0 + g * 8 + j;
                    cv[gi][j] = make_uchar4(0, 0, 0, 0);       // pixels outside: never written
                    if (g < kAllGroups && col_in && y < EMDQ_YE)
                        cv[gi][j] = EMDQ_TGT(canvas)[(size_t)(y + EMDQ_TGT(oy)) * EMDQ_TGT(cpitch4) +
                                                     (x + EMDQ_TGT(ox))];
                }
            }
            for (; b < Bt.count; b = tile_next<PY, PAIRS>(Bt, b, x0, y0), ++it) {
                const int a = it & 1;
                const bool ok = tc::mbar_wait(acc_full + a, (it >> 1) & 1, kWaitLimit, true);
                tc::fence_after_sync();
                if (!ok || *abort_flag) {
                    *abort_flag = 1;
                    alive = false;
                    break;
                }
                if (idle) {
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(acc_empty + a);
                    continue;
                }
                const TcProblem &P = Bt.p[b];
                const uint8_t *__restrict__ frame = M.frame[b];
                const float ra = P.ref[0], rb = P.ref[1], ru = P.ref[2], rv = P.ref[3], rs = P.ref[4];
                const uint32_t lane_base = tmem + a * kTcAccCols + (static_cast<uint32_t>(q * 32) << 16);
#pragma unroll
                for (int gi = 0; gi < kMyGroups; ++gi) {
                    const int g = set + gi * kSets;
                    if (g >= kAllGroups) break;
#pragma unroll
                    for (int h = 0; h < 8; h += 4) {
                        // four rows' channels at a time (the register budget of 20 warps)
                        float F[kTcCh][4];
#pragma unroll
                        for (int ch = 0; ch < kTcCh; ++ch)
                            tc::tmem_ld_x4(lane_base + ch * PY + g * 8 + h, F[ch]);
                        tc::tmem_wait_ld();
                        if (g == g_last && h == 4) {
                            // the accumulator has been read: hand it back to the MMA warp
                            tc::fence_before_sync();
                            __syncwarp();
                            if (lane == 0) tc::mbar_arrive(acc_empty + a);
                        }
                        if (y0 + g * 8 + h >= EMDQ_YE) continue;     // no row of these four is inside
                        // the four displacements first (the channels' registers free
                        // before the taps), then each pixel's sample and update
                        float dx[4], dy[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float py = static_cast<float>(y0 + g * 8 + h + j);
                            dx[j] = NAN;
                            dy[j] = NAN;
                            if (F[5][j] > 0.f) {
                                const float2 d = tc_displacement(F[0][j], F[1][j], F[2][j], F[3][j],
                                                                 F[4][j], F[5][j], ra, rb, ru, rv, rs,
                                                                 px, py);
                                dx[j] = d.x;
                                dy[j] = d.y;
                            }
                        }
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int y = y0 + g * 8 + h + j;
                            Tap t = tap_setup<CH>(EMDQ_TGT(fw), EMDQ_TGT(fh), EMDQ_TGT(pitch), px,
                                                  static_cast<float>(y), dx[j], dy[j]);
                            t.ok = t.ok && col_in && y < EMDQ_YE;
                            // sampled and blended without a branch, the update kept where the sample
                            // is valid (an invalid tap set-up points at the frame's first pixel with
                            // zero weights, so every load stays inside the frame)
                            float v[CH];
                            tap_sample<CH>(frame, t, v);
                            const uchar4 nv = blend_update_r<CH>(cv[gi][h + j], v, rw1_of[cv[gi][h + j].w]);
                            if (t.ok) cv[gi][h + j] = nv;
                        }
                    }
                }
            }
            if (!alive) break;
#pragma unroll
            for (int gi = 0; gi < kMyGroups; ++gi) {
                const int g = set + gi * kSets;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int y = y0 + g * 8 + j;
                    if (g < kAllGroups && col_in && y < EMDQ_YE)
                        EMDQ_TGT(canvas)[(size_t)(y + EMDQ_TGT(oy)) * EMDQ_TGT(cpitch4) +
                                         (x + EMDQ_TGT(ox))] = cv[gi][j];
                }
            }
        }
    }
#undef EMDQ_TGT
#undef EMDQ_YE
    __syncwarp();
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::mbar_wait(done, 0, kWaitLimit, true);
        if (*abort_flag) {
            atomicMax(err, (int)EMDQ_ETIMEOUT);
            for (int k = *consumed; k < *issued; ++k)
                tc::mbar_wait(full + (k % kTcStages), (k / kTcStages) & 1, kWaitLimit, true);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, kTcTmemCols);
}

}  // namespace emdq

using namespace emdq;
using namespace emdq_host;

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

constexpr size_t kErrBytes = 256;

}  // namespace

size_t field_tc_workspace_bytes(int n, int grid_w, int grid_h)
{
    return kErrBytes + tc_operand_bytes_max(n, grid_w, grid_h);
}

namespace {

// Fill problem b of a batch: geometry, tensor maps of its operands (A at ops, B after it),
// the reference-row, column-count and output pointers.  ops must be 256-byte aligned (TMA
// needs 16).
emdq_status tc_problem(TcBatch &Bt, int b, const float *q, const float *c, const float *src, int n,
                       int gx0, int gy0, int gw, int gh, float alpha, float *ref, int *kcount,
                       float2 *disp, char *ops, int py)
{
    auto encode = encode_fn();
    if (!encode) return EMDQ_ECUDA;
    const TcGeom g = tc_geom(n, gw, gh, py);
    if (g.hp / py > 65535 || g.hp > (1 << 24) || g.wp > (1 << 24)) return EMDQ_ENOTSUP;
    auto *A = reinterpret_cast<__nv_bfloat162 *>(ops);
    auto *B = reinterpret_cast<__nv_bfloat162 *>(ops + align_up(g.a_bytes, 1024));
    {
        cuuint64_t dims[2] = {(cuuint64_t)g.kp, (cuuint64_t)g.wp};
        cuuint64_t strides[1] = {(cuuint64_t)g.kp * 2};
        cuuint32_t box[2] = {kTcK, kTcM};
        cuuint32_t estr[2] = {1, 1};
        if (encode(&Bt.tmA[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return EMDQ_ECUDA;
    }
    {
        cuuint64_t dims[3] = {(cuuint64_t)g.kp, (cuuint64_t)g.hp, (cuuint64_t)kTcCh};
        cuuint64_t strides[2] = {(cuuint64_t)g.kp * 2, (cuuint64_t)g.hp * g.kp * 2};
        cuuint32_t box[3] = {kTcK, (cuuint32_t)py, kTcCh};
        cuuint32_t estr[3] = {1, 1, 1};
        if (encode(&Bt.tmB[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, B, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return EMDQ_ECUDA;
    }
    TcProblem &P = Bt.p[b];
    P.q = q;
    P.c = c;
    P.src = reinterpret_cast<const float2 *>(src);
    P.n = n;
    P.kp = g.kp;
    P.gx0 = gx0;
    P.gy0 = gy0;
    P.gw = gw;
    P.gh = gh;
    P.wp = g.wp;
    P.hp = g.hp;
    P.alpha = alpha;
    P.A = A;
    P.B = B;
    P.ref = ref;
    P.kcount = kcount;
    P.disp = disp;
    P.ntx = g.wp / kTcM;
    P.tile0 = b == 0 ? 0 : Bt.p[b - 1].tile0 + Bt.p[b - 1].ntiles;
    P.ntiles = P.ntx * (g.hp / py);
    P.block0 = b == 0 ? 0 : Bt.p[b - 1].block0 + Bt.p[b - 1].nblocks;
    P.a_blocks = g.wp / kPrepRowsA;
    P.nblocks = P.a_blocks + (g.hp + kPrepRowsB - 1) / kPrepRowsB;
    return EMDQ_OK;
}

template <int PY>
cudaError_t tc_set_smem()
{
    return cudaFuncSetAttribute(field_tc_kernel<PY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TcShape<PY>::SmemBytes);
}

template <int PY>
cudaError_t tc_launch_gemm(cudaLaunchConfig_t &cfg, const TcBatch &Bt)
{
    cfg.dynamicSmemBytes = TcShape<PY>::SmemBytes;
    return cudaLaunchKernelEx(&cfg, field_tc_kernel<PY>, Bt);
}

// A programmatic dependent launch of `blocks` CTAs of `threads` on st: its set-up (barriers,
// TMEM) overlaps the tail of the prep launch before it.
cudaLaunchConfig_t pdl_config(int blocks, int threads, cudaStream_t st, cudaLaunchAttribute *at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

// The prep launch and the GEMM launch (a programmatic dependent of the prep) of a batch
// whose problems were filled for tiles of py pixel rows.
emdq_status tc_run(TcBatch &Bt, int py, cudaStream_t st)
{
    const DeviceInfo &D = device_info();
    static std::mutex mu;
    static int attr_dev = -1;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (attr_dev != D.device) {
            if (tc_set_smem<16>() != cudaSuccess || tc_set_smem<24>() != cudaSuccess ||
                tc_set_smem<32>() != cudaSuccess || tc_set_smem<40>() != cudaSuccess)
                return EMDQ_ECUDA;
            attr_dev = D.device;
        }
    }
    const TcProblem &last = Bt.p[Bt.count - 1];
    Bt.total_tiles = last.tile0 + last.ntiles;
    const int blocks = last.block0 + last.nblocks;
    field_tc_prep_kernel<<<blocks, kPrepThreads, 0, st>>>(Bt);
    if (cudaGetLastError() != cudaSuccess) return EMDQ_ECUDA;
    const int grid = Bt.total_tiles < D.sms ? Bt.total_tiles : D.sms;   // persistent: one CTA per SM
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = pdl_config(grid, kTcThreads, st, at);
    cudaError_t e;
    switch (py) {
    case 16: e = tc_launch_gemm<16>(cfg, Bt); break;
    case 24: e = tc_launch_gemm<24>(cfg, Bt); break;
    case 40: e = tc_launch_gemm<40>(cfg, Bt); break;
    default: e = tc_launch_gemm<32>(cfg, Bt); break;
    }
    return e == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

template <int CH, int PY, bool PAIRS = false>
cudaError_t mosaic_launch(cudaLaunchConfig_t &cfg, const TcBatch &Bt, const MosaicBatch &M)
{
    static std::mutex mu;
    static int attr_dev = -1;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (attr_dev != device_info().device) {
            const cudaError_t e = cudaFuncSetAttribute(mosaic_tc_kernel<CH, PY, PAIRS>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)TcShape<PY>::SmemBytes);
            if (e != cudaSuccess) return e;
            attr_dev = device_info().device;
        }
    }
    cfg.dynamicSmemBytes = TcShape<PY>::SmemBytes;
    return cudaLaunchKernelEx(&cfg, mosaic_tc_kernel<CH, PY, PAIRS>, Bt, M);
}

template <int CH>
cudaError_t mosaic_dispatch(int py, cudaLaunchConfig_t &cfg, const TcBatch &Bt, const MosaicBatch &M)
{
    switch (py) {
    case 16: return mosaic_launch<CH, 16>(cfg, Bt, M);
    case 24: return mosaic_launch<CH, 24>(cfg, Bt, M);
    case 32: return mosaic_launch<CH, 32>(cfg, Bt, M);
    default: return mosaic_launch<CH, 40>(cfg, Bt, M);
    }
}

// The prep launch and the fused launch of a group of frames whose problems were filled for
// tiles of py rows; M carries the frames, the canvas and the origin, and gets the union.
// pairs: independent pairs (every problem's canvas and frame geometry in M.tgt, the tiles
// those of each problem's window; tiles of kMosPYDefault rows only).
emdq_status mosaic_run(TcBatch &Bt, MosaicBatch &M, int channels, int py, cudaStream_t st,
                       bool pairs = false)
{
    long long ux0 = 0, uy0 = 0, ux1 = 0, uy1 = 0;
    for (int b = 0; b < (pairs ? 0 : Bt.count); ++b) {
        const TcProblem &P = Bt.p[b];
        const long long x0 = P.gx0, y0 = P.gy0, x1 = x0 + P.gw, y1 = y0 + P.gh;
        ux0 = (b == 0 || x0 < ux0) ? x0 : ux0;
        uy0 = (b == 0 || y0 < uy0) ? y0 : uy0;
        ux1 = (b == 0 || x1 > ux1) ? x1 : ux1;
        uy1 = (b == 0 || y1 > uy1) ? y1 : uy1;
    }
    const long long uw = ux1 - ux0, uh = uy1 - uy0;
    const long long ntx = (uw + kTcM - 1) / kTcM, nty = (uh + py - 1) / py;
    if (ntx * nty > (1 << 30)) return EMDQ_ENOTSUP;
    M.ux0 = (int)ux0;
    M.uy0 = (int)uy0;
    M.uw = (int)uw;
    M.uh = (int)uh;
    M.ntx = (int)ntx;
    M.ntiles = (int)(ntx * nty);
    const TcProblem &last = Bt.p[Bt.count - 1];
    Bt.total_tiles = last.tile0 + last.ntiles;
    if (pairs) {
        if (py != kMosPYDefault) return EMDQ_ENOTSUP;
        M.ntiles = Bt.total_tiles;
    }
    field_tc_prep_kernel<<<last.block0 + last.nblocks, kPrepThreads, 0, st>>>(Bt);
    if (cudaGetLastError() != cudaSuccess) return EMDQ_ECUDA;
    const DeviceInfo &D = device_info();
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = pdl_config(M.ntiles < D.sms ? M.ntiles : D.sms, kMosThreads, st, at);
    const cudaError_t e =
        pairs ? (channels == 3 ? mosaic_launch<3, kMosPYDefault, true>(cfg, Bt, M)
                               : mosaic_launch<1, kMosPYDefault, true>(cfg, Bt, M))
              : (channels == 3 ? mosaic_dispatch<3>(py, cfg, Bt, M) : mosaic_dispatch<1>(py, cfg, Bt, M));
    return e == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

bool tc_device_ok()
{
    const DeviceInfo &D = device_info();
    return D.device >= 0 && D.cc_major == 10 && D.smem_optin >= kTcSmemMax;
}

bool tc_py_ok(int py)
{
    for (int c : kTcPYChoices)
        if (c == py) return true;
    return false;
}

// The tile height chosen for a batch: the autotuner's choice for the batch's size class
// (mean window pixels and mean match count, each to a power of two), else the default.
struct TileChoice {
    int key, py;
};
std::mutex g_tile_mu;
std::vector<TileChoice> g_tile_choices;

int tile_class(const emdq_field_problem *problems, int count)
{
    double px = 0.0, n = 0.0;
    for (int b = 0; b < count; ++b) {
        px += (double)problems[b].grid_w * problems[b].grid_h;
        n += problems[b].n;
    }
    px /= count;
    n /= count;
    const int lp = px > 1.0 ? (int)std::floor(std::log2(px)) : 0;
    const int ln = n > 1.0 ? (int)std::floor(std::log2(n)) : 0;
    return (lp << 8) | (ln << 3) | (count > 7 ? 7 : count);
}

int chosen_tile_rows(int key)
{
    std::lock_guard<std::mutex> lk(g_tile_mu);
    for (const TileChoice &t : g_tile_choices)
        if (t.key == key) return t.py;
    return kTcPYDefault;
}

void record_tile_rows(int key, int py)
{
    std::lock_guard<std::mutex> lk(g_tile_mu);
    for (TileChoice &t : g_tile_choices)
        if (t.key == key) {
            t.py = py;
            return;
        }
    g_tile_choices.push_back({key, py});
}

// Batch workspace: 1024 bytes (error word at 0), then per problem 1024 bytes (reference row
// at 0, column count at 64) and its 1024-aligned operands.
size_t batch_problem_bytes(int n, int gw, int gh)
{
    return 1024 + tc_operand_bytes_max(n, gw, gh);
}

}  // namespace

emdq_status field_tc_launch(const float *q, const float *c, const float *src, int n, int gx0,
                            int gy0, int gw, int gh, float alpha, float *ref, float2 *disp,
                            char *ws, size_t ws_bytes, cudaStream_t st, const MosaicArgs *mos)
{
    if (mos && mos->channels != 1 && mos->channels != 3) return EMDQ_EINVAL;
    const DeviceInfo &D = device_info();
    if (D.device < 0) return EMDQ_ECUDA;
    if (!tc_device_ok()) return EMDQ_ENOTSUP;           // tcgen05: sm_100 family only
    if (ws_bytes < field_tc_workspace_bytes(n, gw, gh)) return EMDQ_EWORKSPACE;
    static thread_local TcBatch Bt;
    Bt.count = 1;
    Bt.err = reinterpret_cast<int *>(ws);
    int *kcount = Bt.err + 1;                 // written by the prep kernel, read by the GEMM
    const int py = mos ? kMosPYDefault : kTcPYDefault;
    const emdq_status rc = tc_problem(Bt, 0, q, c, src, n, gx0, gy0, gw, gh, alpha, ref, kcount,
                                      disp, ws + kErrBytes, py);
    if (rc != EMDQ_OK) return rc;
    if (!mos) return tc_run(Bt, py, st);
    // one frame through the fused group path
    static thread_local MosaicBatch M;
    M.frame[0] = mos->frame;
    M.fw = mos->fw;
    M.fh = mos->fh;
    M.pitch = mos->pitch;
    M.canvas = mos->canvas;
    M.cpitch4 = mos->cpitch4;
    M.ox = mos->ox;
    M.oy = mos->oy;
    return mosaic_run(Bt, M, mos->channels, py, st);
}

extern "C" size_t emdq_field_batch_workspace_size(const emdq_field_problem *problems, int count)
{
    if (!problems || count < 1 || count > kFieldBatchMax) return 0;
    size_t total = 1024;
    for (int b = 0; b < count; ++b) {
        if (problems[b].n < 1 || problems[b].grid_w < 0 || problems[b].grid_h < 0) return 0;
        total += batch_problem_bytes(problems[b].n, problems[b].grid_w, problems[b].grid_h);
    }
    return total;
}

namespace {

emdq_status field_batch_run(const emdq_field_problem *problems, int count, int py, void *workspace,
                            size_t workspace_bytes, void *stream)
{
    if (!problems || count < 1) return EMDQ_EINVAL;
    if (count > kFieldBatchMax || !tc_py_ok(py)) return EMDQ_ENOTSUP;
    for (int b = 0; b < count; ++b) {
        const emdq_field_problem &f = problems[b];
        if (!f.q || !f.c || !f.src || !f.disp_out || f.n < 1 || f.grid_w < 1 || f.grid_h < 1 ||
            !(f.alpha > 0.f) || !std::isfinite(f.alpha))
            return EMDQ_EINVAL;
        if (!aligned(f.q, 16) || !aligned(f.c, 4) || !aligned(f.src, 8) || !aligned(f.disp_out, 8))
            return EMDQ_EINVAL;
    }
    const size_t need = emdq_field_batch_workspace_size(problems, count);
    if (need == 0) return EMDQ_EINVAL;
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return EMDQ_EWORKSPACE;
    if (device_info().device < 0) return EMDQ_ECUDA;
    if (!tc_device_ok()) return EMDQ_ENOTSUP;
    static thread_local TcBatch Bt;
    char *ws = static_cast<char *>(workspace);
    Bt.count = count;
    Bt.err = reinterpret_cast<int *>(ws);
    size_t off = 1024;
    for (int b = 0; b < count; ++b) {
        const emdq_field_problem &f = problems[b];
        float *ref = reinterpret_cast<float *>(ws + off);
        int *kcount = reinterpret_cast<int *>(ws + off + 64);
        const emdq_status rc =
            tc_problem(Bt, b, f.q, f.c, f.src, f.n, f.grid_x0, f.grid_y0, f.grid_w, f.grid_h,
                       f.alpha, ref, kcount, reinterpret_cast<float2 *>(f.disp_out), ws + off + 1024,
                       py);
        if (rc != EMDQ_OK) return rc;
        off += batch_problem_bytes(f.n, f.grid_w, f.grid_h);
    }
    return tc_run(Bt, py, static_cast<cudaStream_t>(stream));
}

}  // namespace

extern "C" emdq_status emdq_field_batch(const emdq_field_problem *problems, int count,
                                        void *workspace, size_t workspace_bytes, void *stream)
{
    if (!problems || count < 1) return EMDQ_EINVAL;
    return field_batch_run(problems, count, chosen_tile_rows(tile_class(problems, count)), workspace,
                           workspace_bytes, stream);
}

extern "C" emdq_status emdq_field_batch_ex(const emdq_field_problem *problems, int count,
                                           int tile_rows, void *workspace, size_t workspace_bytes,
                                           void *stream)
{
    return field_batch_run(problems, count, tile_rows, workspace, workspace_bytes, stream);
}

extern "C" int emdq_field_batch_tile_rows(const emdq_field_problem *problems, int count)
{
    if (!problems || count < 1 || count > kFieldBatchMax) return -1;
    return chosen_tile_rows(tile_class(problems, count));
}

extern "C" emdq_status emdq_field_batch_autotune(const emdq_field_problem *problems, int count,
                                                 void *workspace, size_t workspace_bytes,
                                                 void *stream, int reps, int *tile_rows_out,
                                                 float *ms_out)
{
    if (!problems || count < 1 || reps < 1) return EMDQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return EMDQ_ECUDA;
    }
    emdq_status rc = EMDQ_OK;
    int best_py = kTcPYDefault;
    float best = -1.f;
    for (int py : kTcPYChoices) {
        // one untimed call (operands, caches), then reps timed calls
        rc = field_batch_run(problems, count, py, workspace, workspace_bytes, stream);
        if (rc != EMDQ_OK) break;
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = EMDQ_ECUDA; break; }
        for (int r = 0; r < reps && rc == EMDQ_OK; ++r)
            rc = field_batch_run(problems, count, py, workspace, workspace_bytes, stream);
        if (rc != EMDQ_OK) break;
        float ms = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = EMDQ_ECUDA;
            break;
        }
        ms /= reps;
        if (best < 0.f || ms < best) {
            best = ms;
            best_py = py;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != EMDQ_OK) return rc;
    record_tile_rows(tile_class(problems, count), best_py);
    if (tile_rows_out) *tile_rows_out = best_py;
    if (ms_out) *ms_out = best;
    return EMDQ_OK;
}

// ------------------------------------------------------------------ emdq_mosaic_batch
extern "C" size_t emdq_mosaic_batch_workspace_size(const emdq_mosaic_problem *problems, int count)
{
    if (!problems || count < 1 || count > kFieldBatchMax) return 0;
    size_t total = 1024;
    for (int b = 0; b < count; ++b) {
        if (problems[b].n < 1 || problems[b].grid_w < 0 || problems[b].grid_h < 0) return 0;
        total += batch_problem_bytes(problems[b].n, problems[b].grid_w, problems[b].grid_h);
    }
    return total;
}

extern "C" emdq_status emdq_mosaic_batch_ex(const emdq_mosaic_problem *problems, int count, int fw,
                                            int fh, int channels, int frame_pitch, uint8_t *canvas,
                                            int canvas_w, int canvas_h, int canvas_pitch,
                                            int origin_x, int origin_y, int tile_rows,
                                            void *workspace, size_t workspace_bytes, void *stream)
{
    if (!problems || count < 1 || !canvas || fw < 1 || fh < 1 || (channels != 1 && channels != 3) ||
        frame_pitch < fw * channels || canvas_w < 1 || canvas_h < 1 ||
        canvas_pitch < 4 * canvas_w || canvas_pitch % 4 != 0)
        return EMDQ_EINVAL;
    if (count > kFieldBatchMax || !tc_py_ok(tile_rows)) return EMDQ_ENOTSUP;
    if ((long long)fh * frame_pitch > 0x7fffffffLL) return EMDQ_ENOTSUP;   // 32-bit tap offsets
    if (!aligned(canvas, 4)) return EMDQ_EINVAL;
    for (int b = 0; b < count; ++b) {
        const emdq_mosaic_problem &f = problems[b];
        if (!f.q || !f.c || !f.src || !f.frame || f.n < 1 || f.grid_w < 1 || f.grid_h < 1 ||
            !(f.alpha > 0.f) || !std::isfinite(f.alpha))
            return EMDQ_EINVAL;
        if (!aligned(f.q, 16) || !aligned(f.c, 4) || !aligned(f.src, 8)) return EMDQ_EINVAL;
        if ((long long)f.grid_x0 + origin_x < 0 || (long long)f.grid_y0 + origin_y < 0 ||
            (long long)f.grid_x0 + origin_x + f.grid_w > canvas_w ||
            (long long)f.grid_y0 + origin_y + f.grid_h > canvas_h)
            return EMDQ_EINVAL;
    }
    const size_t need = emdq_mosaic_batch_workspace_size(problems, count);
    if (need == 0) return EMDQ_EINVAL;
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return EMDQ_EWORKSPACE;
    if (device_info().device < 0) return EMDQ_ECUDA;
    if (!tc_device_ok()) return EMDQ_ENOTSUP;
    static thread_local TcBatch Bt;
    static thread_local MosaicBatch M;
    char *ws = static_cast<char *>(workspace);
    Bt.count = count;
    Bt.err = reinterpret_cast<int *>(ws);
    size_t off = 1024;
    for (int b = 0; b < count; ++b) {
        const emdq_mosaic_problem &f = problems[b];
        float *ref = reinterpret_cast<float *>(ws + off);
        int *kcount = reinterpret_cast<int *>(ws + off + 64);
        const emdq_status rc = tc_problem(Bt, b, f.q, f.c, f.src, f.n, f.grid_x0, f.grid_y0,
                                          f.grid_w, f.grid_h, f.alpha, ref, kcount, nullptr,
                                          ws + off + 1024, tile_rows);
        if (rc != EMDQ_OK) return rc;
        M.frame[b] = f.frame;
        off += batch_problem_bytes(f.n, f.grid_w, f.grid_h);
    }
    M.fw = fw;
    M.fh = fh;
    M.pitch = frame_pitch;
    M.canvas = reinterpret_cast<uchar4 *>(canvas);
    M.cpitch4 = canvas_pitch / 4;
    M.ox = origin_x;
    M.oy = origin_y;
    return mosaic_run(Bt, M, channels, tile_rows, static_cast<cudaStream_t>(stream));
}

extern "C" emdq_status emdq_mosaic_batch(const emdq_mosaic_problem *problems, int count, int fw,
                                         int fh, int channels, int frame_pitch, uint8_t *canvas,
                                         int canvas_w, int canvas_h, int canvas_pitch, int origin_x,
                                         int origin_y, void *workspace, size_t workspace_bytes,
                                         void *stream)
{
    return emdq_mosaic_batch_ex(problems, count, fw, fh, channels, frame_pitch, canvas, canvas_w,
                                canvas_h, canvas_pitch, origin_x, origin_y, kMosPYDefault, workspace,
                                workspace_bytes, stream);
}

// ------------------------------------------------------------------ emdq_mosaic_pairs
namespace {

// The bytes of canvas rows a pair may update: from its window's first pixel to its last.
void pair_span(const emdq_mosaic_pair &f, uintptr_t &lo, uintptr_t &hi)
{
    const uintptr_t base = reinterpret_cast<uintptr_t>(f.canvas);
    lo = base + (uintptr_t)((long long)(f.grid_y0 + f.origin_y) * f.canvas_pitch +
                            4LL * (f.grid_x0 + f.origin_x));
    hi = base + (uintptr_t)((long long)(f.grid_y0 + f.origin_y + f.grid_h - 1) * f.canvas_pitch +
                            4LL * (f.grid_x0 + f.origin_x + f.grid_w));
}

}  // namespace

extern "C" size_t emdq_mosaic_pairs_workspace_size(const emdq_mosaic_pair *pairs, int count)
{
    if (!pairs || count < 1 || count > kFieldBatchMax) return 0;
    size_t total = 1024;
    for (int b = 0; b < count; ++b) {
        if (pairs[b].n < 1 || pairs[b].grid_w < 0 || pairs[b].grid_h < 0) return 0;
        total += batch_problem_bytes(pairs[b].n, pairs[b].grid_w, pairs[b].grid_h);
    }
    return total;
}

extern "C" emdq_status emdq_mosaic_pairs(const emdq_mosaic_pair *pairs, int count, int channels,
                                         void *workspace, size_t workspace_bytes, void *stream)
{
    if (!pairs || count < 1 || (channels != 1 && channels != 3)) return EMDQ_EINVAL;
    if (count > kFieldBatchMax) return EMDQ_ENOTSUP;
    for (int b = 0; b < count; ++b) {
        const emdq_mosaic_pair &f = pairs[b];
        if (!f.q || !f.c || !f.src || !f.frame || !f.canvas || f.n < 1 || f.grid_w < 1 ||
            f.grid_h < 1 || !(f.alpha > 0.f) || !std::isfinite(f.alpha) || f.fw < 1 || f.fh < 1 ||
            f.frame_pitch < f.fw * channels || f.canvas_w < 1 || f.canvas_h < 1 ||
            f.canvas_pitch < 4 * f.canvas_w || f.canvas_pitch % 4 != 0)
            return EMDQ_EINVAL;
        if (!aligned(f.q, 16) || !aligned(f.c, 4) || !aligned(f.src, 8) || !aligned(f.canvas, 4))
            return EMDQ_EINVAL;
        if ((long long)f.grid_x0 + f.origin_x < 0 || (long long)f.grid_y0 + f.origin_y < 0 ||
            (long long)f.grid_x0 + f.origin_x + f.grid_w > f.canvas_w ||
            (long long)f.grid_y0 + f.origin_y + f.grid_h > f.canvas_h)
            return EMDQ_EINVAL;
        if ((long long)f.fh * f.frame_pitch > 0x7fffffffLL) return EMDQ_ENOTSUP;   // 32-bit tap offsets
    }
    // the tiles of different pairs run in no fixed order: no two pairs may update the same
    // canvas bytes (checked on the spans of canvas rows their windows cover)
    for (int a = 0; a < count; ++a) {
        uintptr_t alo, ahi;
        pair_span(pairs[a], alo, ahi);
        for (int b = a + 1; b < count; ++b) {
            uintptr_t blo, bhi;
            pair_span(pairs[b], blo, bhi);
            if (alo < bhi && blo < ahi) return EMDQ_EINVAL;
        }
    }
    const size_t need = emdq_mosaic_pairs_workspace_size(pairs, count);
    if (need == 0) return EMDQ_EINVAL;
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return EMDQ_EWORKSPACE;
    if (device_info().device < 0) return EMDQ_ECUDA;
    if (!tc_device_ok()) return EMDQ_ENOTSUP;
    static thread_local TcBatch Bt;
    static thread_local MosaicBatch M;
    char *ws = static_cast<char *>(workspace);
    Bt.count = count;
    Bt.err = reinterpret_cast<int *>(ws);
    size_t off = 1024;
    for (int b = 0; b < count; ++b) {
        const emdq_mosaic_pair &f = pairs[b];
        float *ref = reinterpret_cast<float *>(ws + off);
        int *kcount = reinterpret_cast<int *>(ws + off + 64);
        const emdq_status rc = tc_problem(Bt, b, f.q, f.c, f.src, f.n, f.grid_x0, f.grid_y0,
                                          f.grid_w, f.grid_h, f.alpha, ref, kcount, nullptr,
                                          ws + off + 1024, kMosPYDefault);
        if (rc != EMDQ_OK) return rc;
        M.frame[b] = f.frame;
        MosaicTarget &T = M.tgt[b];
        T.canvas = reinterpret_cast<uchar4 *>(f.canvas);
        T.cpitch4 = f.canvas_pitch / 4;
        T.ox = f.origin_x;
        T.oy = f.origin_y;
        T.fw = f.fw;
        T.fh = f.fh;
        T.pitch = f.frame_pitch;
        off += batch_problem_bytes(f.n, f.grid_w, f.grid_h);
    }
    return mosaic_run(Bt, M, channels, kMosPYDefault, static_cast<cudaStream_t>(stream), true);
}
