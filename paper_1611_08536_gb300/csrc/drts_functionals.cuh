// Device helpers of the Eq. 26/27 extensions, shared by the stand-alone
// kernels (drts_functionals.cu) and the persistent step kernel.
#pragma once

#include <cuda_bf16.h>

#include "drts_device.cuh"

namespace drts {
namespace {

// element offset of canonical state s of right-hand side r in a state buffer
// (for the tensor-core layout: the bf16 element of x0 2^Ex; x1 is 512 further,
// x2 1024)
__device__ __forceinline__ int64_t state_offset(const StepArgs &a, int64_t s, int r)
{
    const int64_t v = s / kDirs;
    const int d = int(s - v * kDirs);
    if (a.tcx) return v * 6144 + (((d >> 3) * 24 + (r >> 3)) * 64) + (r & 7) * 8 + (d & 7);
    if (a.R == 1) return int64_t(d) * a.V + v;
    // batched: groups of four right-hand sides, the four values side by side
    return (int64_t(r >> 2) * a.rhs_stride + int64_t(d) * a.V + v) * 4 + (r & 3);
}

// Point detector d of right-hand side r on x(t) (Eq. 27 with a sparse F):
// the CTA sums the detector's entries, each thread a strided subset in
// entry order, then warp shuffles and one warp over the warp sums, all in a
// fixed order, so the readout is deterministic.  red: >= 32 doubles of
// shared memory.  Every thread of the CTA must call it.
template <class XT, bool COHERENT>
__device__ __forceinline__ void point_detector_block(const StepArgs &a, const XT *x, int r, int d, double *red)
{
    const PointDetectors &P = a.pd;
    const int64_t e1 = P.off[d + 1];
    double acc = 0.0;
    for (int64_t e = P.off[d] + threadIdx.x; e < e1; e += blockDim.x) {
        const int64_t o = state_offset(a, P.state[e], r);
        double xv;
        if (a.tcx) {
            // the value is the sum of its three bf16 terms
            const __nv_bfloat16 *xh = reinterpret_cast<const __nv_bfloat16 *>(x);
            xv = double(__bfloat162float(xh[o])) + double(__bfloat162float(xh[o + 512])) +
                 double(__bfloat162float(xh[o + 1024]));
        } else {
            xv = double(COHERENT ? __ldcg(x + o) : x[o]);
        }
        acc += P.w[e] * xv;
    }
    for (int k = 16; k > 0; k >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, k);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int k = 16; k > 0; k >>= 1) v += __shfl_down_sync(0xffffffffu, v, k);
        if (threadIdx.x == 0) P.hist[int64_t(r) * P.stride_r + a.t * P.n_det + d] = v;
    }
    __syncthreads();
}

}  // namespace
}  // namespace drts
