// Shared device helpers of libemdq (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "emdq.h"

namespace emdq {

// Upper bound of every device-side spin wait (iterations of a ~100 ns back-off): about
// half a second, after which the waiting thread records EMDQ_ETIMEOUT and returns.
constexpr unsigned kSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// 2^x with one MUFU.EX2 (ftz: results below 2^-126 flush to 0, a weight that no sum
// notices next to the nearest match's).
__device__ __forceinline__ float ex2_ftz(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x with one MUFU.RCP (rcp.approx.ftz.f32: within one ulp of the quotient for normal x;
// subnormal x flushes to zero and gives +inf).
__device__ __forceinline__ float rcp_approx_ftz(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Blended planar DQ (a, b, u, v) = (r_w, r_z, d_x, d_y), not normalised, and scale s,
// applied to p: s (R p + t) with R, t of the normalised DQ.  With n2 = a^2 + b^2:
//   cos th = (a^2 - b^2)/n2, sin th = 2ab/n2, t = 2 (a u - b v, b u + a v)/n2
// (the real part is (cos th/2, sin th/2) and t^ = 2 d r*).
__device__ __forceinline__ float2 apply_blend(float a, float b, float u, float v, float s,
                                              float px, float py)
{
    const float inv = 1.0f / (a * a + b * b);
    const float ct = (a * a - b * b) * inv;
    const float st = 2.0f * a * b * inv;
    const float tx = 2.0f * (a * u - b * v) * inv;
    const float ty = 2.0f * (b * u + a * v) * inv;
    return make_float2(s * (ct * px - st * py + tx), s * (st * px + ct * py + ty));
}

// Records the most severe status seen (larger codes are more severe for the ones a
// kernel can raise: ENOCONV < EDEGENERATE ... the host maps them).
__device__ __forceinline__ void raise_status(int *flag, int status)
{
    atomicMax(flag, status);
}

}  // namespace emdq

// Host-side helpers shared by the entry points.
namespace emdq_host {

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct DeviceInfo {
    int device = -1;
    int sms = 0;
    int cc_major = 0, cc_minor = 0;
    size_t smem_optin = 0;
};
// Cached per-device properties (thread-safe, one query per device).
const DeviceInfo &device_info();

}  // namespace emdq_host
