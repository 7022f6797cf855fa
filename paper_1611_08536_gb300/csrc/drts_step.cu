// The DRTS time step x(t+1) = A x(t) + s(t) (Eq. 23 and 26 of
// arXiv:1611.08536) with the detector readout of Eq. 27 and the energy
// ledger fused in.
//
// One warp owns one slice (32 rows: 32 consecutive voxels, one direction m).
// Lane l streams its row's nonzeros four at a time with one 16-byte value load
// and one 8-byte code load; both are lane-interleaved so a warp moves 512 + 256
// contiguous bytes per step of the loop.  A 16-bit code names the column as
// (neighbour offset, direction); a shared-memory table turns it into the
// distance to the column in the state vector, which is stored direction-major
// (x[n*V + v]) so that the 32 lanes of a slice gather 32 consecutive floats.
// The matrix is read with streaming (evict-first) loads; the state is read
// through the read-only cache.
#include <cuda_runtime.h>

#include "drts_device.cuh"

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

// VT: stored value type; XT: state type; AT: accumulation type
template <class VT, class XT, class AT>
__global__ void __launch_bounds__(256) step_kernel(StepArgs a)
{
    __shared__ int32_t s_delta[kCodes];
    __shared__ double s_ledger[2];
    __shared__ SourceEntry s_src[kMaxSrc];
    __shared__ double s_src_val[kMaxSrc];

    const int64_t V = a.V;
    for (int c = threadIdx.x; c < kCodes; c += blockDim.x) {
        const int d = c / kDirs, n = c % kDirs;
        s_delta[c] = int32_t(n * V + (int64_t(d / 9 - 1) * a.ny + (d / 3 % 3 - 1)) * a.nx + (d % 3 - 1));
    }
    if (threadIdx.x < 2) s_ledger[threadIdx.x] = 0.0;
    for (int e = threadIdx.x; e < a.n_src; e += blockDim.x) {
        s_src[e] = a.src[e];
        const SourceProfile &p = a.prof[a.src[e].prof];
        double val = 0.0;
        if (a.step_scale) val = a.src[e].w * a.step_scale[a.src[e].rhs];
        else if (a.t >= p.t0 && a.t < p.t0 + p.n_t) val = a.src[e].w * a.prof_vals[p.off + (a.t - p.t0)];
        s_src_val[e] = val;
    }
    __syncthreads();

    const XT *__restrict__ x = static_cast<const XT *>(a.x);
    XT *__restrict__ y = static_cast<XT *>(a.y);
    const VT *__restrict__ vals = static_cast<const VT *>(a.A.vals);
    const uint16_t *__restrict__ codes = a.A.codes;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int nxy = a.nx * a.ny;
    AT ab_lane = 0, ex_lane = 0;

    for (int64_t q = warp0; q < a.A.n_slices; q += nwarps) {
        const int64_t b = q / kDirs;
        const int m = int(q - b * kDirs);
        const int64_t v = b * kSlice + lane;
        const int len4 = a.A.slice_len4[q];
        const int64_t base = a.A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup;
        AT acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
#pragma unroll 4
        for (int g = 0; g < len4; ++g) {
            AT w[4];
            int c[4];
            const int64_t idx = base + int64_t(g) * (kSlice * kGroup);
            load4(vals + idx, w);
            load_codes(codes + idx, c);
            acc0 += w[0] * AT(__ldg(x + (v + s_delta[c[0]])));
            acc1 += w[1] * AT(__ldg(x + (v + s_delta[c[1]])));
            acc2 += w[2] * AT(__ldg(x + (v + s_delta[c[2]])));
            acc3 += w[3] * AT(__ldg(x + (v + s_delta[c[3]])));
        }
        AT acc = (acc0 + acc1) + (acc2 + acc3);
        if (a.A.row_scale) acc *= AT(a.A.row_scale[q * kSlice + lane]);
        if (v < V) {
            const int64_t row = int64_t(m) * V + v;
            for (int e = 0; e < a.n_src; ++e)
                if (s_src[e].slice == q && s_src[e].lane == lane) acc += AT(s_src_val[e]);
            y[row] = XT(acc);
            // column functionals of x(t): absorbed, exited, detector (Eq. 27)
            const AT xs = AT(x[row]);
            const int k = a.med[v];
            ab_lane += AT(a.tab.absorb[k]) * xs;
            const int xx = int(v % a.nx), yy = int(v / a.nx % a.ny), zz = int(v / nxy);
            const int bx = xx == 0 ? 0 : (xx == a.nx - 1 ? 2 : 1);
            const int by = yy == 0 ? 0 : (yy == a.ny - 1 ? 2 : 1);
            const int bz = zz == 0 ? 0 : (zz == a.nz - 1 ? 2 : 1);
            const int mask = bz * 9 + by * 3 + bx;
            if (mask != 13) {
                const int ti = (k * 27 + mask) * kDirs + m;
                ex_lane += AT(a.tab.exit_total[ti]) * xs;
                const double ed = a.tab.exit_det[ti];
                if (ed > 0.0 && a.det) {
                    // patch coordinates (u, v) = the two other axes in x, y, z order
                    const int fa = a.det_face >> 1;
                    const int cu = fa == 0 ? yy : xx, nu = fa == 0 ? a.ny : a.nx;
                    const int cv = fa == 2 ? yy : zz, nv = fa == 2 ? a.ny : a.nz;
                    const int p = int(int64_t(cv) * a.det_nv / nv) * a.det_nu +
                                  int(int64_t(cu) * a.det_nu / nu);
                    atomicAdd(a.det + p, ed * double(xs));
                }
            }
        }
    }
    const AT ab_w = warp_sum(ab_lane), ex_w = warp_sum(ex_lane);
    if (lane == 0) {
        atomicAdd(&s_ledger[0], double(ab_w));
        atomicAdd(&s_ledger[1], double(ex_w));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_ledger[0] != 0.0) atomicAdd(&a.ledger[2], s_ledger[0]);
        if (s_ledger[1] != 0.0) atomicAdd(&a.ledger[3], s_ledger[1]);
        if (blockIdx.x == 0) {          // injected mass, once per step
            double inj = 0.0;
            for (int e = 0; e < a.n_src; ++e) inj += s_src_val[e];
            if (inj != 0.0) atomicAdd(&a.ledger[1], inj);
        }
    }
}

template <class XT>
__global__ void to_canonical_kernel(const XT *x, int64_t V, int R, int r, double *out)
{
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= V * kDirs) return;
    const int64_t v = s / kDirs;
    const int d = int(s % kDirs);
    out[s] = double(x[(int64_t(d) * V + v) * R + r]);
}

template <class XT>
__global__ void from_canonical_kernel(const double *in, int64_t V, int R, int r, XT *x)
{
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= V * kDirs) return;
    const int64_t v = s / kDirs;
    const int d = int(s % kDirs);
    x[(int64_t(d) * V + v) * R + r] = XT(in[s]);
}

template <class XT>
__global__ void sum_kernel(const XT *x, int64_t n, int R, int r, double *out)
{
    double acc = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        acc += double(x[i * R + r]);
    acc = warp_sum(acc);
    __shared__ double s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) atomicAdd(out, t);
    }
}

}  // namespace

int step_default_blocks(int precision, int R, int threads)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (precision == DRTS_FP64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel<double, double, double>, threads, 0);
    else if (precision == DRTS_FP32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel<float, float, float>, threads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel<__half, float, float>, threads, 0);
    (void)R;
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

cudaError_t launch_step(const StepArgs &a, int blocks, int threads, cudaStream_t s)
{
    if (a.A.precision == DRTS_FP64) step_kernel<double, double, double><<<blocks, threads, 0, s>>>(a);
    else if (a.A.precision == DRTS_FP32) step_kernel<float, float, float><<<blocks, threads, 0, s>>>(a);
    else step_kernel<__half, float, float><<<blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_to_canonical(const void *x, int precision, int64_t V, int R, int r,
                                double *out, cudaStream_t s)
{
    const int th = 256;
    const unsigned blocks = unsigned((V * kDirs + th - 1) / th);
    if (precision == DRTS_FP64) to_canonical_kernel<<<blocks, th, 0, s>>>(static_cast<const double *>(x), V, R, r, out);
    else to_canonical_kernel<<<blocks, th, 0, s>>>(static_cast<const float *>(x), V, R, r, out);
    return cudaGetLastError();
}

cudaError_t launch_from_canonical(const double *in, int precision, int64_t V, int R, int r,
                                  void *x, cudaStream_t s)
{
    const int th = 256;
    const unsigned blocks = unsigned((V * kDirs + th - 1) / th);
    if (precision == DRTS_FP64) from_canonical_kernel<<<blocks, th, 0, s>>>(in, V, R, r, static_cast<double *>(x));
    else from_canonical_kernel<<<blocks, th, 0, s>>>(in, V, R, r, static_cast<float *>(x));
    return cudaGetLastError();
}

cudaError_t launch_ledger_sum(const void *x, int precision, int64_t n, int R, int r,
                              double *out, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (precision == DRTS_FP64) sum_kernel<<<sms * 2, 256, 0, s>>>(static_cast<const double *>(x), n, R, r, out);
    else sum_kernel<<<sms * 2, 256, 0, s>>>(static_cast<const float *>(x), n, R, r, out);
    return cudaGetLastError();
}

}  // namespace drts
