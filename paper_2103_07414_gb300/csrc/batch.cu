// emdq_batch: the whole hot path for a batch of independent pairs in one call -- learned
// warm start (optional), all EMDQ fits in one cooperative launch, then per group of up to 16
// pairs their BF16 fields and warps fused in one operand + tensor-core launch pair
// (emdq_mosaic_pairs), or, for a group whose pairs update overlapping canvas rows or differ
// in channels, the fields of the group in one launch pair followed by each pair's warp in
// pair order -- all on the caller's stream, with every scratch buffer in one workspace.
#include "common.cuh"

using namespace emdq_host;

namespace {

constexpr int kBatchMax = 64;            // the batched fit's limit
constexpr int kFieldGroup = 16;          // the batched field's limit

size_t al(size_t v) { return align_up(v, 256); }

struct BatchLayout {
    size_t p0, fit, field, disp, total;  // offsets; field and disp reused by every group
};

// p0[count] (if warm), the fit workspace, then the largest group's field workspace and
// displacement fields.
bool batch_layout(const emdq_pair *pairs, int count, bool warm, BatchLayout &L)
{
    size_t off = 0;
    L.p0 = off;
    if (warm)
        for (int b = 0; b < count; ++b) off += al(sizeof(float) * (size_t)pairs[b].n);
    emdq_fit_problem fp[kBatchMax];
    for (int b = 0; b < count; ++b) fp[b].n = pairs[b].n;
    const size_t fit = emdq_fit_batch_workspace_size(fp, count);
    if (fit == 0) return false;
    L.fit = off;
    off += al(fit);
    size_t field = 0, disp = 0;
    for (int g0 = 0; g0 < count; g0 += kFieldGroup) {
        const int gc = count - g0 < kFieldGroup ? count - g0 : kFieldGroup;
        emdq_field_problem f[kFieldGroup];
        size_t d = 0;
        for (int i = 0; i < gc; ++i) {
            const emdq_pair &p = pairs[g0 + i];
            f[i].n = p.n;
            f[i].grid_w = p.grid_w;
            f[i].grid_h = p.grid_h;
            d += al(sizeof(float) * 2 * (size_t)p.grid_w * (size_t)p.grid_h);
        }
        const size_t w = emdq_field_batch_workspace_size(f, gc);
        if (w == 0) return false;
        field = w > field ? w : field;
        disp = d > disp ? d : disp;
    }
    L.field = off;
    off += al(field);
    L.disp = off;
    off += al(disp);
    L.total = off;
    return true;
}

}  // namespace

extern "C" size_t emdq_batch_workspace_size(const emdq_pair *pairs, int count, int warm)
{
    if (!pairs || count < 1 || count > kBatchMax) return 0;
    for (int b = 0; b < count; ++b)
        if (pairs[b].n < 0 || pairs[b].grid_w < 0 || pairs[b].grid_h < 0) return 0;
    BatchLayout L;
    return batch_layout(pairs, count, warm != 0, L) ? L.total : 0;
}

extern "C" emdq_status emdq_batch_ex(const emdq_pair *pairs, int count, const emdq_params *prm,
                                     const float *warm_params, const int *fit_ctas,
                                     const int *fit_phases, int nphases, void *workspace,
                                     size_t workspace_bytes, void *stream)
{
    if (!pairs || count < 1) return EMDQ_EINVAL;
    if (fit_phases && fit_ctas) return EMDQ_EINVAL;     // a phased batch splits on its own
    if (count > kBatchMax) return EMDQ_ENOTSUP;
    for (int b = 0; b < count; ++b) {
        const emdq_pair &p = pairs[b];
        if (!p.frame || !p.canvas || p.grid_w < 1 || p.grid_h < 1) return EMDQ_EINVAL;
    }
    const bool warm = warm_params != nullptr;
    BatchLayout L;
    if (!batch_layout(pairs, count, warm, L)) return EMDQ_EINVAL;
    if (!workspace || workspace_bytes < L.total || !aligned(workspace, 256)) return EMDQ_EWORKSPACE;
    char *ws = static_cast<char *>(workspace);
    emdq_params P;
    emdq_default_params(&P);
    if (prm) P = *prm;

    // 1. learned warm start (Sec. II's EM started from predicted inlier weights)
    float *p0[kBatchMax] = {};
    if (warm) {
        const float *src[kBatchMax], *dst[kBatchMax];
        int n[kBatchMax];
        size_t off = L.p0;
        for (int b = 0; b < count; ++b) {
            src[b] = pairs[b].src;
            dst[b] = pairs[b].dst;
            n[b] = pairs[b].n;
            p0[b] = reinterpret_cast<float *>(ws + off);
            off += al(sizeof(float) * (size_t)pairs[b].n);
        }
        const emdq_status rc = emdq_warm_start(src, dst, n, p0, count, warm_params, stream);
        if (rc != EMDQ_OK) return rc;
    }
    // 2. every EMDQ fit in one cooperative launch
    {
        emdq_fit_problem fp[kBatchMax];
        for (int b = 0; b < count; ++b) {
            const emdq_pair &p = pairs[b];
            fp[b] = emdq_fit_problem{p.src, p.dst, p.n, p.frame_w, p.frame_h, p0[b],
                                     p.q_out, p.c_out, p.p_out, p.info};
        }
        const emdq_status rc =
            fit_phases ? emdq_fit_batch_phases(fp, count, &P, fit_phases, nphases, ws + L.fit,
                                               L.field - L.fit, stream)
                       : emdq_fit_batch_ex(fp, count, &P, fit_ctas, ws + L.fit, L.field - L.fit, stream);
        if (rc != EMDQ_OK) return rc;
    }
    // 3. per group of up to 16 pairs: fields and warps fused; or the fields in one launch
    //    pair, then their warps in pair order
    for (int g0 = 0; g0 < count; g0 += kFieldGroup) {
        const int gc = count - g0 < kFieldGroup ? count - g0 : kFieldGroup;
        {
            emdq_mosaic_pair m[kFieldGroup];
            bool same_ch = true;
            for (int i = 0; i < gc; ++i) {
                const emdq_pair &p = pairs[g0 + i];
                const float alpha = P.alpha > 0.f ? P.alpha : emdq_alpha_for_frame(p.frame_w, p.frame_h);
                m[i] = emdq_mosaic_pair{p.q_out, p.c_out, p.src, p.n, p.grid_x0, p.grid_y0,
                                        p.grid_w, p.grid_h, alpha, p.frame, p.frame_w, p.frame_h,
                                        p.frame_pitch, p.canvas, p.canvas_w, p.canvas_h,
                                        p.canvas_pitch, p.origin_x, p.origin_y};
                same_ch = same_ch && p.channels == pairs[g0].channels;
            }
            if (same_ch) {
                // argument refusals (EINVAL: overlapping canvas rows among others; ENOTSUP)
                // come before any launch: the group then takes the unfused calls
                const emdq_status rc =
                    emdq_mosaic_pairs(m, gc, pairs[g0].channels, ws + L.field, L.disp - L.field, stream);
                if (rc == EMDQ_OK) continue;
                if (rc != EMDQ_EINVAL && rc != EMDQ_ENOTSUP) return rc;
            }
        }
        emdq_field_problem f[kFieldGroup];
        size_t off = L.disp;
        for (int i = 0; i < gc; ++i) {
            const emdq_pair &p = pairs[g0 + i];
            const float alpha = P.alpha > 0.f ? P.alpha : emdq_alpha_for_frame(p.frame_w, p.frame_h);
            f[i] = emdq_field_problem{p.q_out, p.c_out, p.src, p.n, p.grid_x0, p.grid_y0,
                                      p.grid_w, p.grid_h, alpha, reinterpret_cast<float *>(ws + off)};
            off += al(sizeof(float) * 2 * (size_t)p.grid_w * (size_t)p.grid_h);
        }
        emdq_status rc = emdq_field_batch(f, gc, ws + L.field, L.disp - L.field, stream);
        if (rc != EMDQ_OK) return rc;
        for (int i = 0; i < gc; ++i) {
            const emdq_pair &p = pairs[g0 + i];
            rc = mosaic_warp(p.frame, p.frame_w, p.frame_h, p.channels, p.frame_pitch,
                             f[i].disp_out, p.grid_x0, p.grid_y0, p.grid_w, p.grid_h, p.canvas,
                             p.canvas_w, p.canvas_h, p.canvas_pitch, p.origin_x, p.origin_y,
                             stream);
            if (rc != EMDQ_OK) return rc;
        }
    }
    return EMDQ_OK;
}

extern "C" emdq_status emdq_batch(const emdq_pair *pairs, int count, const emdq_params *prm,
                                  const float *warm_params, const int *fit_ctas, void *workspace,
                                  size_t workspace_bytes, void *stream)
{
    return emdq_batch_ex(pairs, count, prm, warm_params, fit_ctas, nullptr, 0, workspace,
                         workspace_bytes, stream);
}
