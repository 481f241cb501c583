// Mosaic warp + blend (Sec. III-F, Eqs. 23-24 as read): a gather over the canvas window.
// HBM-bound: per window pixel one 8-byte field read, one 4-byte canvas read and write
// (colour + merge weight packed in one aligned word) and the bilinear taps of the frame,
// which neighbouring threads share through L1/L2 because the field is smooth.
#include "common.cuh"

namespace emdq {

constexpr int kWarpThreadsX = 128;

__device__ __forceinline__ unsigned blend_channel(unsigned c, float w, float v, float w1)
{
    // c <- clamp(floor((w c + v)/(w + 1) + 1/2), 0, 255).  w c + v is exact for integer
    // v and the quotient is correctly rounded, so ties land exactly on .5 as in FP64.
    const float z = floorf(__fdiv_rn(fmaf(w, static_cast<float>(c), v), w1) + 0.5f);
    return static_cast<unsigned>(fminf(fmaxf(z, 0.f), 255.f));
}

template <int CH>
__global__ void __launch_bounds__(kWarpThreadsX) mosaic_warp_kernel(
    const uint8_t *__restrict__ frame, int fw, int fh, int pitch,
    const float2 *__restrict__ disp, int gx0, int gy0, int gw, int gh,
    uchar4 *__restrict__ canvas, int cpitch4, int ox, int oy)
{
    const int x = blockIdx.x * kWarpThreadsX + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= gw) return;
    const float2 d = __ldcs(disp + (size_t)y * gw + x);
    // u = p + d in FP32 (one rounding): the coverage and tap decisions
    const float ux = __fadd_rn(static_cast<float>(gx0 + x), d.x);
    const float uy = __fadd_rn(static_cast<float>(gy0 + y), d.y);
    if (!(ux >= 0.f && ux <= static_cast<float>(fw - 1) && uy >= 0.f &&
          uy <= static_cast<float>(fh - 1)))
        return;
    const int x0 = static_cast<int>(floorf(ux)), y0 = static_cast<int>(floorf(uy));
    const float fx = ux - static_cast<float>(x0), fy = uy - static_cast<float>(y0);
    const int x1 = min(x0 + 1, fw - 1), y1 = min(y0 + 1, fh - 1);
    const float w00 = (1.f - fx) * (1.f - fy), w10 = fx * (1.f - fy);
    const float w01 = (1.f - fx) * fy, w11 = fx * fy;
    const uint8_t *r0 = frame + (size_t)y0 * pitch;
    const uint8_t *r1 = frame + (size_t)y1 * pitch;
    uchar4 *cp = canvas + (size_t)(gy0 + y + oy) * cpitch4 + (gx0 + x + ox);
    uchar4 cv = *cp;
    const float w = static_cast<float>(cv.w);
    const float w1 = w + 1.f;
    float v[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        v[k] = w00 * __ldg(r0 + x0 * CH + k) + w10 * __ldg(r0 + x1 * CH + k) +
               w01 * __ldg(r1 + x0 * CH + k) + w11 * __ldg(r1 + x1 * CH + k);
    }
    cv.x = blend_channel(cv.x, w, v[0], w1);
    if (CH == 3) {
        cv.y = blend_channel(cv.y, w, v[1 % CH], w1);
        cv.z = blend_channel(cv.z, w, v[2 % CH], w1);
    }
    cv.w = static_cast<unsigned char>(cv.w < 30 ? cv.w + 1 : 30);
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
    if (grid_w == 0 || grid_h == 0) return EMDQ_OK;      // empty window: nothing to read
    if (!disp || !aligned(disp, 8) || !aligned(canvas, 4)) return EMDQ_EINVAL;
    if ((long long)grid_x0 + origin_x < 0 || (long long)grid_y0 + origin_y < 0 ||
        (long long)grid_x0 + origin_x + grid_w > canvas_w ||
        (long long)grid_y0 + origin_y + grid_h > canvas_h)
        return EMDQ_EINVAL;
    if (grid_h > 65535) return EMDQ_ENOTSUP;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dim3 grid((grid_w + kWarpThreadsX - 1) / kWarpThreadsX, grid_h);
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
