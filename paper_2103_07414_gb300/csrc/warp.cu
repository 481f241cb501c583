// Mosaic warp + blend (Sec. III-F, Eqs. 23-24 as read): a gather over the canvas window.
// HBM-bound: per window pixel one 8-byte field read, one 4-byte canvas read and write
// (colour + merge weight packed in one aligned word) and the bilinear taps of the frame,
// which neighbouring threads share through L1/L2 because the field is smooth.
#include "blend.cuh"
#include "common.cuh"

namespace emdq {

constexpr int kWarpThreadsX = 128;

// Each thread blends kWarpPix pixels of one row (x = x0 + threadIdx.x + k * kWarpThreadsX,
// coalesced for every k), issuing all their loads before any update so several gathers
// are in flight per thread.
constexpr int kWarpPix = 4;

template <int CH>
__global__ void __launch_bounds__(kWarpThreadsX) mosaic_warp_kernel(
    const uint8_t *__restrict__ frame, int fw, int fh, int pitch,
    const float2 *__restrict__ disp, int gx0, int gy0, int gw, int gh,
    uchar4 *__restrict__ canvas, int cpitch4, int ox, int oy)
{
    const int y = blockIdx.y;
    const int xb = blockIdx.x * (kWarpThreadsX * kWarpPix) + threadIdx.x;
    float2 d[kWarpPix];
#pragma unroll
    for (int k = 0; k < kWarpPix; ++k) {
        const int x = xb + k * kWarpThreadsX;
        d[k] = x < gw ? __ldcs(disp + (size_t)y * gw + x) : make_float2(NAN, NAN);
    }
    Tap t[kWarpPix];
    uchar4 cv[kWarpPix];
    uchar4 *cp[kWarpPix];
#pragma unroll
    for (int k = 0; k < kWarpPix; ++k) {
        const int x = xb + k * kWarpThreadsX;
        t[k] = tap_setup<CH>(fw, fh, pitch, static_cast<float>(gx0 + x), static_cast<float>(gy0 + y),
                             d[k].x, d[k].y);
        cp[k] = canvas + (size_t)(gy0 + y + oy) * cpitch4 + (gx0 + x + ox);
        if (t[k].ok) cv[k] = *cp[k];
    }
    float v[kWarpPix][CH];
#pragma unroll
    for (int k = 0; k < kWarpPix; ++k)
        if (t[k].ok) tap_sample<CH>(frame, t[k], v[k]);
#pragma unroll
    for (int k = 0; k < kWarpPix; ++k)
        if (t[k].ok) *cp[k] = blend_update<CH>(cv[k], v[k]);
}

// G frames of a sequence blended in one pass (held to 51 registers for G <= 4: ten blocks
// of 128 threads per SM hide more of the gather latency than the few spilled words cost):
// the thread of canvas pixel p applies frames
// 0..G-1 to p in order, exactly as G mosaic_warp launches would (the blend of a pixel
// depends only on that pixel's earlier updates), but reads and writes the canvas word
// once, and issues the field loads and bilinear taps of all G frames before any update, so
// their memory latencies overlap.  Threads cover the union of the G windows.
constexpr int kWarpBatchMax = 8;

struct WarpFrame {
    const uint8_t *frame;
    const float2 *disp;
    int gx0, gy0, gw, gh;
};

struct WarpBatch {
    WarpFrame f[kWarpBatchMax];
};

template <int CH, int G>
__global__ void __launch_bounds__(kWarpThreadsX, G <= 4 ? 10 : 1) mosaic_warp_batch_kernel(
    const __grid_constant__ WarpBatch W, int fw, int fh, int pitch, int ux0, int uy0, int uw,
    uchar4 *__restrict__ canvas, int cpitch4, int ox, int oy)
{
    const int x = ux0 + blockIdx.x * kWarpThreadsX + threadIdx.x;   // reference coordinates
    const int y = uy0 + blockIdx.y;
    if (x >= ux0 + uw) return;
    Tap t[G];
    bool any = false;
#pragma unroll
    for (int k = 0; k < G; ++k) {
        const WarpFrame &F = W.f[k];
        const int lx = x - F.gx0, ly = y - F.gy0;
        float2 d = make_float2(NAN, NAN);
        if (lx >= 0 && lx < F.gw && ly >= 0 && ly < F.gh) d = __ldcs(F.disp + (size_t)ly * F.gw + lx);
        t[k] = tap_setup<CH>(fw, fh, pitch, static_cast<float>(x), static_cast<float>(y), d.x, d.y);
        any = any || t[k].ok;
    }
    if (!any) return;
    uchar4 *cp = canvas + (size_t)(y + oy) * cpitch4 + (x + ox);
    uchar4 cv = *cp;
    float v[G][CH];
#pragma unroll
    for (int k = 0; k < G; ++k)
        if (t[k].ok) tap_sample<CH>(W.f[k].frame, t[k], v[k]);
#pragma unroll
    for (int k = 0; k < G; ++k)
        if (t[k].ok) cv = blend_update<CH>(cv, v[k]);
    *cp = cv;
}

template <int CH>
__global__ void insert_reference_kernel(const uint8_t *__restrict__ frame, int fw, int fh,
                                        int pitch, uchar4 *__restrict__ canvas, int cpitch4,
                                        int ox, int oy)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= fw) return;
    const uint8_t *f = frame + (size_t)y * pitch + (size_t)x * CH;
    uchar4 cv;
    cv.x = f[0];
    cv.y = CH == 3 ? f[1 % CH] : 0;
    cv.z = CH == 3 ? f[2 % CH] : 0;
    cv.w = 1;
    canvas[(size_t)(y + oy) * cpitch4 + x + ox] = cv;
}

}  // namespace emdq

using namespace emdq;
using namespace emdq_host;

extern "C" emdq_status mosaic_warp(const uint8_t *frame, int fw, int fh, int channels,
                                   int frame_pitch, const float *disp, int grid_x0,
                                   int grid_y0, int grid_w, int grid_h, uint8_t *canvas,
                                   int canvas_w, int canvas_h, int canvas_pitch, int origin_x,
                                   int origin_y, void *stream)
{
    if (!frame || !canvas || fw < 1 || fh < 1 || (channels != 1 && channels != 3) ||
        frame_pitch < fw * channels || grid_w < 0 || grid_h < 0 || canvas_w < 1 ||
        canvas_h < 1 || canvas_pitch < 4 * canvas_w || canvas_pitch % 4 != 0)
        return EMDQ_EINVAL;
    if ((long long)fh * frame_pitch > 0x7fffffffLL) return EMDQ_ENOTSUP;   // 32-bit tap offsets
    if (grid_w == 0 || grid_h == 0) return EMDQ_OK;      // empty window: nothing to read
    if (!disp || !aligned(disp, 8) || !aligned(canvas, 4)) return EMDQ_EINVAL;
    if ((long long)grid_x0 + origin_x < 0 || (long long)grid_y0 + origin_y < 0 ||
        (long long)grid_x0 + origin_x + grid_w > canvas_w ||
        (long long)grid_y0 + origin_y + grid_h > canvas_h)
        return EMDQ_EINVAL;
    if (grid_h > 65535) return EMDQ_ENOTSUP;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dim3 grid((grid_w + kWarpThreadsX * kWarpPix - 1) / (kWarpThreadsX * kWarpPix), grid_h);
    auto *cv = reinterpret_cast<uchar4 *>(canvas);
    const auto *d = reinterpret_cast<const float2 *>(disp);
    if (channels == 3)
        mosaic_warp_kernel<3><<<grid, kWarpThreadsX, 0, st>>>(
            frame, fw, fh, frame_pitch, d, grid_x0, grid_y0, grid_w, grid_h, cv,
            canvas_pitch / 4, origin_x, origin_y);
    else
        mosaic_warp_kernel<1><<<grid, kWarpThreadsX, 0, st>>>(
            frame, fw, fh, frame_pitch, d, grid_x0, grid_y0, grid_w, grid_h, cv,
            canvas_pitch / 4, origin_x, origin_y);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

extern "C" emdq_status mosaic_insert_reference(const uint8_t *frame, int fw, int fh,
                                               int channels, int frame_pitch, uint8_t *canvas,
                                               int canvas_w, int canvas_h, int canvas_pitch,
                                               int origin_x, int origin_y, void *stream)
{
    if (!frame || !canvas || fw < 1 || fh < 1 || (channels != 1 && channels != 3) ||
        frame_pitch < fw * channels || canvas_pitch < 4 * canvas_w || canvas_pitch % 4 != 0 ||
        origin_x < 0 || origin_y < 0 || origin_x + fw > canvas_w || origin_y + fh > canvas_h)
        return EMDQ_EINVAL;
    if (!aligned(canvas, 4)) return EMDQ_EINVAL;
    if (fh > 65535) return EMDQ_ENOTSUP;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dim3 grid((fw + 127) / 128, fh);
    auto *cv = reinterpret_cast<uchar4 *>(canvas);
    if (channels == 3)
        insert_reference_kernel<3><<<grid, 128, 0, st>>>(frame, fw, fh, frame_pitch, cv,
                                                         canvas_pitch / 4, origin_x, origin_y);
    else
        insert_reference_kernel<1><<<grid, 128, 0, st>>>(frame, fw, fh, frame_pitch, cv,
                                                         canvas_pitch / 4, origin_x, origin_y);
    return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}

namespace {
template <int CH, int G>
cudaError_t launch_warp_batch(const WarpBatch &W, dim3 grid, cudaStream_t st, int fw, int fh,
                              int pitch, int ux0, int uy0, int uw, uchar4 *cv, int cpitch4, int ox,
                              int oy)
{
    mosaic_warp_batch_kernel<CH, G><<<grid, kWarpThreadsX, 0, st>>>(W, fw, fh, pitch, ux0, uy0, uw, cv,
                                                                    cpitch4, ox, oy);
    return cudaGetLastError();
}

template <int CH>
cudaError_t dispatch_warp_batch(int count, const WarpBatch &W, dim3 grid, cudaStream_t st, int fw,
                                int fh, int pitch, int ux0, int uy0, int uw, uchar4 *cv, int cpitch4,
                                int ox, int oy)
{
    switch (count) {
    case 1: return launch_warp_batch<CH, 1>(W, grid, st, fw, fh, pitch, ux0, uy0, uw, cv, cpitch4, ox, oy);
    case 2: return launch_warp_batch<CH, 2>(W, grid, st, fw, fh, pitch, ux0, uy0, uw, cv, cpitch4, ox, oy);
    case 3: return launch_warp_batch<CH, 3>(W, grid, st, fw, fh, pitch, ux0, uy0, uw, cv, cpitch4, ox, oy);
    case 4: return launch_warp_batch<CH, 4>(W, grid, st, fw, fh, pitch, ux0, uy0, uw, cv, cpitch4, ox, oy);
    case 5: return launch_warp_batch<CH, 5>(W, grid, st, fw, fh, pitch, ux0, uy0, uw, cv, cpitch4, ox, oy);
    case 6: return launch_warp_batch<CH, 6>(W, grid, st, fw, fh, pitch, ux0, uy0, uw, cv, cpitch4, ox, oy);
    case 7: return launch_warp_batch<CH, 7>(W, grid, st, fw, fh, pitch, ux0, uy0, uw, cv, cpitch4, ox, oy);
    default: return launch_warp_batch<CH, 8>(W, grid, st, fw, fh, pitch, ux0, uy0, uw, cv, cpitch4, ox, oy);
    }
}
}  // namespace

extern "C" emdq_status mosaic_warp_batch(const mosaic_frame *frames, int count, int fw, int fh,
                                         int channels, int frame_pitch, uint8_t *canvas,
                                         int canvas_w, int canvas_h, int canvas_pitch, int origin_x,
                                         int origin_y, void *stream)
{
    if (!frames || count < 1 || !canvas || fw < 1 || fh < 1 || (channels != 1 && channels != 3) ||
        frame_pitch < fw * channels || canvas_w < 1 || canvas_h < 1 ||
        canvas_pitch < 4 * canvas_w || canvas_pitch % 4 != 0)
        return EMDQ_EINVAL;
    if (count > kWarpBatchMax) return EMDQ_ENOTSUP;
    if ((long long)fh * frame_pitch > 0x7fffffffLL) return EMDQ_ENOTSUP;   // 32-bit tap offsets
    if (!aligned(canvas, 4)) return EMDQ_EINVAL;
    WarpBatch W = {};
    long long ux0 = 0, uy0 = 0, ux1 = 0, uy1 = 0;
    int used = 0;
    for (int k = 0; k < count; ++k) {
        const mosaic_frame &f = frames[k];
        if (!f.frame || f.grid_w < 0 || f.grid_h < 0) return EMDQ_EINVAL;
        if (f.grid_w == 0 || f.grid_h == 0) continue;      // empty window: nothing to blend
        if (!f.disp || !aligned(f.disp, 8)) return EMDQ_EINVAL;
        if ((long long)f.grid_x0 + origin_x < 0 || (long long)f.grid_y0 + origin_y < 0 ||
            (long long)f.grid_x0 + origin_x + f.grid_w > canvas_w ||
            (long long)f.grid_y0 + origin_y + f.grid_h > canvas_h)
            return EMDQ_EINVAL;
        W.f[used] = WarpFrame{f.frame, reinterpret_cast<const float2 *>(f.disp), f.grid_x0,
                              f.grid_y0, f.grid_w, f.grid_h};
        const long long x0 = f.grid_x0, y0 = f.grid_y0, x1 = x0 + f.grid_w, y1 = y0 + f.grid_h;
        if (used == 0) {
            ux0 = x0; uy0 = y0; ux1 = x1; uy1 = y1;
        } else {
            ux0 = x0 < ux0 ? x0 : ux0;
            uy0 = y0 < uy0 ? y0 : uy0;
            ux1 = x1 > ux1 ? x1 : ux1;
            uy1 = y1 > uy1 ? y1 : uy1;
        }
        ++used;
    }
    if (used == 0) return EMDQ_OK;
    const int uw = (int)(ux1 - ux0), uh = (int)(uy1 - uy0);
    if (uh > 65535) return EMDQ_ENOTSUP;
    const dim3 grid((uw + kWarpThreadsX - 1) / kWarpThreadsX, uh);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto *cv = reinterpret_cast<uchar4 *>(canvas);
    const cudaError_t e =
        channels == 3 ? dispatch_warp_batch<3>(used, W, grid, st, fw, fh, frame_pitch, (int)ux0,
                                               (int)uy0, uw, cv, canvas_pitch / 4, origin_x, origin_y)
                      : dispatch_warp_batch<1>(used, W, grid, st, fw, fh, frame_pitch, (int)ux0,
                                               (int)uy0, uw, cv, canvas_pitch / 4, origin_x, origin_y);
    return e == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
}
