// Library-level entry points of libemdq: parameters, status strings, device properties and
// the emdq_field dispatcher.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "field.cuh"
#include "field_tc.cuh"

namespace emdq_host {

const DeviceInfo &device_info()
{
    static std::mutex mu;
    static DeviceInfo cache[64];
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        static DeviceInfo none;
        return none;
    }
    std::lock_guard<std::mutex> g(mu);
    DeviceInfo &d = cache[dev];
    if (d.device != dev) {
        cudaDeviceProp p;
        if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
            static DeviceInfo none;
            return none;
        }
        d.sms = p.multiProcessorCount;
        d.cc_major = p.major;
        d.cc_minor = p.minor;
        d.smem_optin = p.sharedMemPerBlockOptin;
        d.device = dev;
    }
    return d;
}

}  // namespace emdq_host

using namespace emdq;
using namespace emdq_host;

extern "C" void emdq_default_params(emdq_params *prm)
{
    if (!prm) return;
    prm->alpha = 0.f;
    prm->max_iters = 20;
    prm->tol_p = 1e-3f;
    prm->sigma2_floor = 0.25f;
    for (int k = 0; k < 4; ++k) prm->reserved[k] = 0;
}

extern "C" float emdq_alpha_for_frame(int w, int h)
{
    // Sec. III-G: alpha = 2e-4 / s^2, s = (w/480 + h/270)/2
    const double s = (w / 480.0 + h / 270.0) / 2.0;
    return static_cast<float>(2e-4 / (s * s));
}

extern "C" float emdq_beta_for_frame(int w, int h)
{
    // Sec. III-G: beta = 3e-3 / s^2, the same resolution scale as alpha
    const double s = (w / 480.0 + h / 270.0) / 2.0;
    return static_cast<float>(3e-3 / (s * s));
}

extern "C" int emdq_abi_version(void) { return EMDQ_ABI_VERSION; }

extern "C" const char *emdq_status_string(int status)
{
    switch (status) {
    case EMDQ_OK: return "ok";
    case EMDQ_EINVAL: return "invalid argument";
    case EMDQ_EDEGENERATE: return "degenerate fit (no weight or no spread)";
    case EMDQ_ENOCONV: return "EM iteration cap reached (outputs valid)";
    case EMDQ_ETIMEOUT: return "bounded device wait gave up";
    case EMDQ_ECUDA: return "CUDA runtime error";
    case EMDQ_EWORKSPACE: return "workspace missing or too small";
    case EMDQ_ENOTSUP: return "unsupported size, precision or device";
    case EMDQ_ENONFINITE: return "non-finite input coordinate";
    default: return "unknown status";
    }
}

namespace {
constexpr size_t kRefBytes = 256;   // reference row, kept at the start of every workspace
}

extern "C" size_t emdq_field_workspace_size(int n, int grid_w, int grid_h, int precision)
{
    if (n < 0 || grid_w < 0 || grid_h < 0) return 0;
    if (precision == EMDQ_FP32) return kRefBytes;
    if (precision == EMDQ_BF16) return kRefBytes + field_tc_workspace_bytes(n, grid_w, grid_h);
    return 0;
}

extern "C" emdq_status emdq_field(const float *q, const float *c, const float *src, int n,
                                  int grid_x0, int grid_y0, int grid_w, int grid_h, float alpha,
                                  int precision, float *disp_out, void *workspace,
                                  size_t workspace_bytes, void *stream)
{
    if (!q || !c || !src || !disp_out || n < 1 || grid_w < 0 || grid_h < 0 || !(alpha > 0.f) ||
        !std::isfinite(alpha))
        return EMDQ_EINVAL;
    if (!aligned(q, 16) || !aligned(src, 8) || !aligned(disp_out, 8)) return EMDQ_EINVAL;
    if (precision != EMDQ_FP32 && precision != EMDQ_BF16) return EMDQ_ENOTSUP;
    const size_t need = emdq_field_workspace_size(n, grid_w, grid_h, precision);
    if (need == 0) return EMDQ_ENOTSUP;
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return EMDQ_EWORKSPACE;
    if (grid_w == 0 || grid_h == 0) return EMDQ_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *ref = static_cast<float *>(workspace);
    if (precision == EMDQ_FP32) {
        field_ref_kernel<<<1, kRefThreads, 0, st>>>(q, c, n, ref);
        if ((grid_h + 7) / 8 > 65535) return EMDQ_ENOTSUP;
        dim3 grid((grid_w + 31) / 32, (grid_h + 7) / 8);
        field_direct_kernel<<<grid, kDirectThreads, 0, st>>>(
            q, c, reinterpret_cast<const float2 *>(src), n, grid_x0, grid_y0, grid_w, grid_h,
            alpha, ref, reinterpret_cast<float2 *>(disp_out));
        return cudaGetLastError() == cudaSuccess ? EMDQ_OK : EMDQ_ECUDA;
    }
    return field_tc_launch(q, c, src, n, grid_x0, grid_y0, grid_w, grid_h, alpha, ref,
                           reinterpret_cast<float2 *>(disp_out),
                           static_cast<char *>(workspace) + kRefBytes, workspace_bytes - kRefBytes,
                           st);
}

extern "C" emdq_status emdq_mosaic(const float *q, const float *c, const float *src, int n,
                                   int grid_x0, int grid_y0, int grid_w, int grid_h, float alpha,
                                   const uint8_t *frame, int fw, int fh, int channels,
                                   int frame_pitch, uint8_t *canvas, int canvas_w, int canvas_h,
                                   int canvas_pitch, int origin_x, int origin_y, void *workspace,
                                   size_t workspace_bytes, void *stream)
{
    if (!q || !c || !src || n < 1 || grid_w < 0 || grid_h < 0 || !(alpha > 0.f) ||
        !std::isfinite(alpha))
        return EMDQ_EINVAL;
    if (!frame || !canvas || fw < 1 || fh < 1 || (channels != 1 && channels != 3) ||
        frame_pitch < fw * channels || canvas_w < 1 || canvas_h < 1 ||
        canvas_pitch < 4 * canvas_w || canvas_pitch % 4 != 0)
        return EMDQ_EINVAL;
    if (!aligned(q, 16) || !aligned(src, 8) || !aligned(canvas, 4)) return EMDQ_EINVAL;
    if ((long long)fh * frame_pitch > 0x7fffffffLL) return EMDQ_ENOTSUP;   // 32-bit tap offsets
    const size_t need = emdq_field_workspace_size(n, grid_w, grid_h, EMDQ_BF16);
    if (need == 0) return EMDQ_ENOTSUP;
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return EMDQ_EWORKSPACE;
    if (grid_w == 0 || grid_h == 0) return EMDQ_OK;
    if ((long long)grid_x0 + origin_x < 0 || (long long)grid_y0 + origin_y < 0 ||
        (long long)grid_x0 + origin_x + grid_w > canvas_w ||
        (long long)grid_y0 + origin_y + grid_h > canvas_h)
        return EMDQ_EINVAL;
    MosaicArgs m;
    m.frame = frame;
    m.fw = fw;
    m.fh = fh;
    m.pitch = frame_pitch;
    m.channels = channels;
    m.canvas = reinterpret_cast<uchar4 *>(canvas);
    m.cpitch4 = canvas_pitch / 4;
    m.ox = origin_x;
    m.oy = origin_y;
    return field_tc_launch(q, c, src, n, grid_x0, grid_y0, grid_w, grid_h, alpha,
                           static_cast<float *>(workspace), nullptr,
                           static_cast<char *>(workspace) + kRefBytes, workspace_bytes - kRefBytes,
                           static_cast<cudaStream_t>(stream), &m);
}
