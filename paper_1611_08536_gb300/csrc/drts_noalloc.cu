// drts_state_sum_noalloc: the state-mass reduction of the energy ledger for
// callers that cannot allocate device memory.
//
// drts_read_detectors gets sum(x(t)) from a reduction whose result buffer it
// allocates with cudaMallocAsync and fills with atomics.  Some callers cannot
// call cudaMalloc at that point: a real-time loop that must not take the
// allocator's locks or wait on its latency, or a process whose device memory
// is owned and budgeted by another runtime's pool.  This entry point computes
// the same sum into memory the caller already owns, keeping its intermediate
// per-block partial sums in a fixed static device array.
//
// The array (kPartials doubles, 32 KiB) lives in every GPU that loads the
// library until the process exits.  All calls share it, so two calls whose
// kernels overlap on the GPU (for example on two streams) race on it; calls
// on one stream are ordered and safe.  Both kernels write every partial they
// later read, so no part of the array needs to start at zero.
#include <cuda_runtime.h>

#include <mutex>

#include "drts_device.cuh"

namespace drts {
namespace {

constexpr int kPartials = 4096;              // one double per block
constexpr int64_t kChunk = 65536;            // states reduced by one block
constexpr int kThreads = 256;

static __device__ __align__(256) double g_partials[kPartials];

template <class XT>
__global__ void __launch_bounds__(kThreads) chunk_sum_kernel(const XT *x, int64_t n, int R, int r,
                                                             double *partials)
{
    const int64_t begin = int64_t(blockIdx.x) * kChunk;
    const int64_t end = begin + kChunk < n ? begin + kChunk : n;
    double acc = 0.0;
    for (int64_t i = begin + threadIdx.x; i < end; i += kThreads) acc += double(x[i * R + r]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double s[kThreads / 32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += s[w];
        partials[blockIdx.x] = t;
    }
}

// fixed-order final reduction of the partials (one block)
__global__ void __launch_bounds__(kThreads) partials_sum_kernel(const double *partials, int nb, double *out)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) acc += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double s[kThreads / 32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += s[w];
        *out = t;
    }
}

// Device address of g_partials for each device, looked up once per device
// with that device current and kept for the life of the process (a device
// reset would invalidate it; the header tells callers not to reset a device
// they use this entry point on).  The host-side name of the array is only a
// stand-in and must never be passed to a kernel.
std::mutex g_mu;
double *g_addr[64] = {};

cudaError_t partials_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

int64_t noalloc_max_states() { return int64_t(kPartials) * kChunk; }

cudaError_t launch_state_sum_noalloc(const void *x, int precision, int64_t n, int R, int r,
                                     double *out, cudaStream_t s)
{
    double *partials = nullptr;
    cudaError_t e = partials_address(&partials);
    if (e != cudaSuccess) return e;
    const int nb = int((n + kChunk - 1) / kChunk);
    if (nb > 0) {
        if (precision == DRTS_FP64)
            chunk_sum_kernel<<<nb, kThreads, 0, s>>>(static_cast<const double *>(x), n, R, r, partials);
        else
            chunk_sum_kernel<<<nb, kThreads, 0, s>>>(static_cast<const float *>(x), n, R, r, partials);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    partials_sum_kernel<<<1, kThreads, 0, s>>>(partials, nb, out);
    return cudaGetLastError();
}

}  // namespace drts
