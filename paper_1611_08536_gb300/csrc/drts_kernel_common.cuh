// Device helpers shared by the step kernels (drts_step.cu, drts_batched.cu).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace drts {
namespace {

__device__ __forceinline__ void load4(const float *p, float v[4])
{
    const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const double *p, double v[4])
{
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load4(const __half *p, float v[4])
{
    const uint2 t = __ldcs(reinterpret_cast<const uint2 *>(p));
    const __half2 a = *reinterpret_cast<const __half2 *>(&t.x);
    const __half2 b = *reinterpret_cast<const __half2 *>(&t.y);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
}
__device__ __forceinline__ void load4_smem(const float *p, float v[4])
{
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4_smem(const double *p, double v[4])
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load4_smem(const __half *p, float v[4])
{
    const uint2 t = *reinterpret_cast<const uint2 *>(p);
    const float2 fa = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
    const float2 fb = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
    v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
}
__device__ __forceinline__ void load_codes_smem(const uint16_t *p, int c[4])
{
    const uint2 t = *reinterpret_cast<const uint2 *>(p);
    c[0] = int(t.x & 0xffffu); c[1] = int(t.x >> 16);
    c[2] = int(t.y & 0xffffu); c[3] = int(t.y >> 16);
}
__device__ __forceinline__ void load_codes(const uint16_t *p, int c[4])
{
    const uint2 t = __ldcs(reinterpret_cast<const uint2 *>(p));
    c[0] = int(t.x & 0xffffu); c[1] = int(t.x >> 16);
    c[2] = int(t.y & 0xffffu); c[3] = int(t.y >> 16);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}


}  // namespace
}  // namespace drts
