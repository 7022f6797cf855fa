// Extensions of the step's source and detector terms (arXiv:1611.08536):
//
//  * point detectors - Eq. 27 with a general sparse F: detector d reads
//    sum_e w_e x_t[s_e] over chosen (voxel, direction) states, every step,
//    into a history like the face-patch detector's;
//  * sub-step sources - Section 4.1 asks for the source function to be
//    sampled in sub-intervals shorter than the step; a population emitted in
//    sub-interval j travels only part of the step, so it lands spread over
//    the column of a partial-path matrix.  Those entries are too many for the
//    step kernels' per-row source test, so a small kernel adds them to
//    y(t+1) after the product;
//  * sensor response - Eq. 27's impulse response h over a window of +-w
//    steps, applied to a recorded detector history.
#include <cuda_runtime.h>

#include "drts_device.cuh"
#include "drts_functionals.cuh"

namespace drts {
namespace {

template <class XT>
__global__ void __launch_bounds__(128) point_det_kernel(StepArgs a)
{
    __shared__ double red[32];
    point_detector_block<XT, false>(a, static_cast<const XT *>(a.x), int(blockIdx.y), int(blockIdx.x), red);
}

__device__ __forceinline__ double bulk_value(const StepArgs &a, const BulkEntry &e)
{
    const SourceProfile &p = a.bulk.prof[e.prof];
    if (a.t >= p.t0 && a.t < p.t0 + p.n_t) return e.w * a.bulk.prof_vals[p.off + (a.t - p.t0)];
    return 0.0;
}

// One CTA: thread g adds group g's sub-step contributions to y(t+1) (groups
// own distinct (state, rhs) pairs, so there are no write conflicts); then
// thread r adds the injected mass of right-hand side r to the ledger, in
// group order (deterministic).  Runs after the product on the same stream.
template <class XT>
__global__ void __launch_bounds__(256) bulk_source_kernel(StepArgs a)
{
    XT *y = static_cast<XT *>(a.y);
    const BulkSources &B = a.bulk;
    for (int g = threadIdx.x; g < B.n_groups; g += blockDim.x) {
        const BulkGroup G = B.groups[g];
        double add = 0.0;
        for (int e = 0; e < G.count; ++e) add += bulk_value(a, B.entries[G.first + e]);
        if (add != 0.0) {
            const int64_t o = state_offset(a, G.state, G.rhs);
            y[o] = XT(double(y[o]) + add);
        }
    }
    for (int r = threadIdx.x; r < a.R; r += blockDim.x) {
        double inj = 0.0;
        for (int g = B.rhs_off[r]; g < B.rhs_off[r + 1]; ++g) {
            const BulkGroup G = B.groups[g];
            for (int e = 0; e < G.count; ++e) inj += bulk_value(a, B.entries[G.first + e]);
        }
        if (inj != 0.0) a.ledger[4 * r + 1] += inj;
    }
}

// M[t - t_begin][d] = sum over k in [t - w, t + w] and [0, t_rec) of
// h[t - k + w] D[k][d]; products and sums rounded separately, in k order.
__global__ void sensor_kernel(const double *D, int64_t t_rec, int n_det, int64_t t_begin, int64_t t_end, int w,
                              const double *h, double *M)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= (t_end - t_begin) * n_det) return;
    const int64_t t = t_begin + i / n_det;
    const int d = int(i % n_det);
    double acc = 0.0;
    for (int64_t k = t - w; k <= t + w; ++k) {
        if (k < 0 || k >= t_rec) continue;
        acc = __dadd_rn(acc, __dmul_rn(h[t - k + w], D[k * n_det + d]));
    }
    M[i] = acc;
}

}  // namespace

cudaError_t launch_point_detectors(const StepArgs &a, cudaStream_t s)
{
    if (a.pd.n_det <= 0 || !a.pd.hist) return cudaSuccess;
    const dim3 grid(unsigned(a.pd.n_det), unsigned(a.R));
    if (a.A.precision == DRTS_FP64) point_det_kernel<double><<<grid, 128, 0, s>>>(a);
    else point_det_kernel<float><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bulk_sources(const StepArgs &a, cudaStream_t s)
{
    if (a.bulk.n_groups <= 0) return cudaSuccess;
    if (a.A.precision == DRTS_FP64) bulk_source_kernel<double><<<1, 256, 0, s>>>(a);
    else bulk_source_kernel<float><<<1, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sensor_response(const double *D, int64_t t_rec, int n_det, int64_t t_begin, int64_t t_end,
                                   int w, const double *h, double *M, cudaStream_t s)
{
    const int64_t n = (t_end - t_begin) * n_det;
    if (n <= 0) return cudaSuccess;
    sensor_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(D, t_rec, n_det, t_begin, t_end, w, h, M);
    return cudaGetLastError();
}

}  // namespace drts
