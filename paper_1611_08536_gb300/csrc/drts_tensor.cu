// Tensor-core form of the batched step X(t+1) = A X(t) + S(t).
//
// The rows of one voxel j (26 directions m) gather only from the 27
// neighbouring voxels i = j + d, so
//     Y[j][m][r] = sum_d sum_n B_{j,d}[m][n] X[j+d][n][r],
// a sum of 27 small dense products (26 x 26 blocks, about 30 % nonzero, times
// a 26 x R state tile).  Each is run on the tensor cores with
// mma.sync.m16n8k16 (bf16 inputs, FP32 accumulation): m and n are padded to
// 32 (two 16-row tiles, two 16-deep k steps), R to a multiple of 8.
//
// Precision: bf16 keeps 8 significant bits.  Each stored FP32 value of A is
// split exactly into three bf16 terms a0 + a1 + a2, the state into a high
// and a low part x0 + x1, and the product is formed as
//     (a0 + a1 + a2) x0 + (a0 + a1) x1,
// exact in A and carrying ~16 bits of x (the dropped terms are below 2^-24 of
// the result).  An approximate A would drift: the stencil is the same for
// every interior voxel, so its rounding error is systematic (a two-term split
// of A drifted 5e-5 in 40 steps).  bf16 has the FP32 exponent range, which
// the state needs (its values span some twenty decades).  The tensor cores'
// FP32 accumulation drops low bits on large additions (plain accumulation of
// the whole row drifted ~3e-7 per step), so each dominant a0 x0 product
// (one k-tile) lands in a fresh fragment and is added to a Kahan-compensated
// sum on the CUDA cores; the correction terms, 2^-8 smaller, accumulate in
// the tensor cores.
//
// Layouts.  A: per (j, d) twelve fragments (m-tile, k-tile, term), each
// 32 lanes x 16 bytes in the register order of the mma A operand, so a warp
// loads a block with coalesced 16-byte loads per lane.  State:
// X[v][r][k] (k = direction padded to 32), so the two k-adjacent values a lane
// needs for a B register are one 8-byte load.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "drts_device.cuh"
#include "drts_kernel_common.cuh"

namespace drts {
namespace {

constexpr int kTcK = 32;

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem)
{
    const __nv_bfloat16 a = __float2bfloat16_rn(lo_elem), b = __float2bfloat16_rn(hi_elem);
    return uint32_t(__bfloat16_as_ushort(a)) | (uint32_t(__bfloat16_as_ushort(b)) << 16);
}

// high and low bf16 parts of two consecutive k values
__device__ __forceinline__ void split2(float2 v, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v.x), h1 = __float2bfloat16_rn(v.y);
    hi = uint32_t(__bfloat16_as_ushort(h0)) | (uint32_t(__bfloat16_as_ushort(h1)) << 16);
    lo = pack_bf16(v.x - __bfloat162float(h0), v.y - __bfloat162float(h1));
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint4 &a, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

__device__ __forceinline__ double tc_source_value(const StepArgs &a, const SourceEntry &e)
{
    if (a.step_scale) return e.w * a.step_scale[e.rhs];
    const SourceProfile &p = a.prof[e.prof];
    if (a.t >= p.t0 && a.t < p.t0 + p.n_t) return e.w * a.prof_vals[p.off + (a.t - p.t0)];
    return 0.0;
}

__device__ __forceinline__ bool tc_in_grid(const StepArgs &a, int jx, int jy, int jz, int d)
{
    const int ix = jx + d % 3 - 1, iy = jy + d / 3 % 3 - 1, iz = jz + d / 9 - 1;
    return ix >= 0 && iy >= 0 && iz >= 0 && ix < a.nx && iy < a.ny && iz < a.nz;
}

// the six fragments (m-tile, term) of k-tile kt of voxel j's block d
__device__ __forceinline__ void tc_load_a(const uint4 *jb, int d, int kt, uint4 A[2][3])
{
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int term = 0; term < 3; ++term) A[mt][term] = __ldcs(jb + (size_t(d) * 12 + (mt * 2 + kt) * 3 + term) * 32);
}

// One warp per (voxel j, group of NT*8 right-hand sides); R/(NT*8) warps share
// a voxel's blocks (they run side by side, so the second read hits L1/L2).
template <int NT>
__global__ void __launch_bounds__(256) tc_step_kernel(StepArgs a, int Rp)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, p = lane & 3;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int groups = Rp / (NT * 8);
    const float *__restrict__ x = static_cast<const float *>(a.x);
    float *__restrict__ y = static_cast<float *>(a.y);
    const uint4 *__restrict__ blocks = a.tc_blocks;
    const int nxy = a.nx * a.ny;

    for (int64_t w = warp0; w < a.V * groups; w += nwarps) {
        const int64_t j = w / groups;
        const int r0 = int(w % groups) * NT * 8;
        const int jx = int(j % a.nx), jy = int(j / a.nx % a.ny), jz = int(j / nxy);
        // big: the a0 x0 products, one fresh fragment per (d, k-tile), added to a
        // Kahan-compensated sum on the CUDA cores; small: the correction terms
        // (below 2^-8 of the result), accumulated in the tensor cores
        float sum[2][NT][4], comp[2][NT][4], small[2][NT][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) sum[mt][nt][q] = comp[mt][nt][q] = small[mt][nt][q] = 0.0f;
        // neighbours inside the grid, in order; the A fragments of the next
        // (neighbour, k-tile) load while the current ones are in use
        const uint4 *jb = blocks + size_t(j) * kOffs * 12 * 32 + lane;
        int d = 0;
        while (d < kOffs && !tc_in_grid(a, jx, jy, jz, d)) ++d;
        uint4 An[2][3];
        if (d < kOffs) tc_load_a(jb, d, 0, An);
        while (d < kOffs) {
            int dn = d + 1;
            while (dn < kOffs && !tc_in_grid(a, jx, jy, jz, dn)) ++dn;
            const int64_t i = j + (int64_t(d / 9 - 1) * a.ny + (d / 3 % 3 - 1)) * a.nx + (d % 3 - 1);
            const float *xi = x + (size_t(i) * Rp + r0) * kTcK;
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) {
                uint4 A[2][3];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int term = 0; term < 3; ++term) A[mt][term] = An[mt][term];
                if (kt == 0) tc_load_a(jb, d, 1, An);
                else if (dn < kOffs) tc_load_a(jb, dn, 0, An);
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const float *xr = xi + (nt * 8 + g) * kTcK + kt * 16 + 2 * p;
                    const float2 v0 = __ldg(reinterpret_cast<const float2 *>(xr));
                    const float2 v1 = __ldg(reinterpret_cast<const float2 *>(xr + 8));
                    uint32_t b0h, b0l, b1h, b1l;
                    split2(v0, b0h, b0l);
                    split2(v1, b1h, b1l);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma_bf16(small[mt][nt], A[mt][2], b0h, b1h);
                        mma_bf16(small[mt][nt], A[mt][1], b0l, b1l);
                        mma_bf16(small[mt][nt], A[mt][1], b0h, b1h);
                        mma_bf16(small[mt][nt], A[mt][0], b0l, b1l);
                        float big[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                        mma_bf16(big, A[mt][0], b0h, b1h);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float yv = big[q] - comp[mt][nt][q];
                            const float t = sum[mt][nt][q] + yv;
                            comp[mt][nt][q] = (t - sum[mt][nt][q]) - yv;
                            sum[mt][nt][q] = t;
                        }
                    }
                }
            }
            d = dn;
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) sum[mt][nt][q] += small[mt][nt][q] - comp[mt][nt][q];
        // sources of this voxel
        for (int e = 0; e < (a.src_voxel[j] ? a.n_src : 0); ++e) {
            const SourceEntry se = a.src[e];
            const int64_t sv = (int64_t(se.slice) / kDirs) * kSlice + se.lane;
            if (sv != j || se.rhs < r0 || se.rhs >= r0 + NT * 8) continue;
            const int sm = int(se.slice % kDirs);
            const float val = float(tc_source_value(a, se));
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int m = mt * 16 + g + (q >> 1) * 8;
                        const int r = r0 + nt * 8 + 2 * p + (q & 1);
                        if (m == sm && r == se.rhs) sum[mt][nt][q] += val;
                    }
        }
        // y[j][r][m], only m < 26 (rows 26..31 of the padding stay zero)
        float *yj = y + (size_t(j) * Rp + r0) * kTcK;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int m = mt * 16 + g + (q >> 1) * 8;
                    const int r = nt * 8 + 2 * p + (q & 1);
                    if (m < kDirs) yj[r * kTcK + m] = sum[mt][nt][q];
                }
    }
}

// Ledger of X(t) in the tensor-core layout: a warp walks (voxel, rhs) rows of
// 32 directions with a stride that is a multiple of Rp, so its right-hand
// side is fixed; lanes accumulate in registers and each warp adds its two
// sums to the block's, then the block's to the FP64 ledger.
__global__ void __launch_bounds__(256) tc_ledger_kernel(StepArgs a, int Rp)
{
    __shared__ double red[2][kMaxRhs];
    for (int i = threadIdx.x; i < 2 * kMaxRhs; i += blockDim.x) (&red[0][0])[i] = 0.0;
    __syncthreads();
    const float *x = static_cast<const float *>(a.x);
    const int lane = threadIdx.x & 31;
    const int64_t rows = a.V * Rp;
    const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;     // a multiple of Rp
    const int r = int(w0 % Rp);
    float ab = 0.0f, ex = 0.0f;
    if (r < a.R && lane < kDirs) {
        for (int64_t row = w0; row < rows; row += nw) {
            const float xs = x[row * kTcK + lane];
            if (xs == 0.0f) continue;
            const int64_t v = row / Rp;
            const int k = a.med[v];
            ab += float(a.tab.absorb[k]) * xs;
            const int xx = int(v % a.nx), yy = int(v / a.nx % a.ny), zz = int(v / (int64_t(a.nx) * a.ny));
            const int mask = (zz == 0 ? 0 : (zz == a.nz - 1 ? 2 : 1)) * 9 +
                             (yy == 0 ? 0 : (yy == a.ny - 1 ? 2 : 1)) * 3 + (xx == 0 ? 0 : (xx == a.nx - 1 ? 2 : 1));
            if (mask != 13) ex += float(a.tab.exit_total[(k * 27 + mask) * kDirs + lane]) * xs;
        }
    }
    ab = warp_sum(ab);
    ex = warp_sum(ex);
    if (lane == 0 && r < a.R) {
        atomicAdd(&red[0][r], double(ab));
        atomicAdd(&red[1][r], double(ex));
    }
    __syncthreads();
    for (int q = threadIdx.x; q < a.R; q += blockDim.x) {
        if (red[0][q] != 0.0) atomicAdd(&a.ledger[4 * q + 2], red[0][q]);
        if (red[1][q] != 0.0) atomicAdd(&a.ledger[4 * q + 3], red[1][q]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int e = 0; e < a.n_src; ++e) {
            const double val = tc_source_value(a, a.src[e]);
            if (val != 0.0) atomicAdd(&a.ledger[4 * a.src[e].rhs + 1], val);
        }
}

// Detector readout of X(t) in the tensor-core layout (one block per patch,
// one thread per rhs, fixed summation order).
__global__ void tc_det_kernel(StepArgs a, int Rp)
{
    const int p = blockIdx.x, r = threadIdx.x;
    if (r >= a.R) return;
    const int fa = a.det_face >> 1, high = a.det_face & 1;
    const int N[3] = {a.nx, a.ny, a.nz};
    const int ua = fa == 0 ? 1 : 0, va = fa == 2 ? 1 : 2;
    const int pu = p % a.det_nu, pv = p / a.det_nu;
    const int Nu = N[ua], Nv = N[va];
    const int u0 = (pu * Nu + a.det_nu - 1) / a.det_nu, u1 = ((pu + 1) * Nu + a.det_nu - 1) / a.det_nu;
    const int v0 = (pv * Nv + a.det_nv - 1) / a.det_nv, v1 = ((pv + 1) * Nv + a.det_nv - 1) / a.det_nv;
    const float *x = static_cast<const float *>(a.x);
    double sum = 0.0;
    for (int cv = v0; cv < v1; ++cv)
        for (int cu = u0; cu < u1; ++cu) {
            int c[3];
            c[fa] = high ? N[fa] - 1 : 0;
            c[ua] = cu;
            c[va] = cv;
            const int64_t v = (int64_t(c[2]) * a.ny + c[1]) * a.nx + c[0];
            const int k = a.med[v];
            const int mask = (c[2] == 0 ? 0 : (c[2] == a.nz - 1 ? 2 : 1)) * 9 +
                             (c[1] == 0 ? 0 : (c[1] == a.ny - 1 ? 2 : 1)) * 3 +
                             (c[0] == 0 ? 0 : (c[0] == a.nx - 1 ? 2 : 1));
            const float *xv = x + (size_t(v) * Rp + r) * kTcK;
            for (int d = 0; d < kDirs; ++d) {
                const double ed = a.tab.exit_det[(k * 27 + mask) * kDirs + d];
                if (ed > 0.0) sum += ed * double(xv[d]);
            }
        }
    a.det[r * a.det_stride_r + p] = sum;
}

__global__ void tc_to_canonical_kernel(const float *x, int64_t V, int Rp, int r, double *out)
{
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= V * kDirs) return;
    const int64_t v = s / kDirs;
    const int d = int(s % kDirs);
    out[s] = double(x[(size_t(v) * Rp + r) * kTcK + d]);
}

__global__ void tc_from_canonical_kernel(const double *in, int64_t V, int Rp, int r, float *x)
{
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= V * kDirs) return;
    const int64_t v = s / kDirs;
    const int d = int(s % kDirs);
    x[(size_t(v) * Rp + r) * kTcK + d] = float(in[s]);
}

__global__ void tc_sum_kernel(const float *x, int64_t V, int Rp, int r, double *out)
{
    double acc = 0.0;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < V * kDirs;
         s += int64_t(gridDim.x) * blockDim.x)
        acc += double(x[(size_t(s / kDirs) * Rp + r) * kTcK + s % kDirs]);
    acc = warp_sum(acc);
    __shared__ double sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) atomicAdd(out, t);
    }
}

template <int NT>
int tc_fit(int threads)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tc_step_kernel<NT>, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace

int tc_rhs_stride(int n_rhs)
{
    int rp = 8;
    while (rp < n_rhs) rp *= 2;
    return rp;
}

// right-hand sides per warp (a multiple of 8, at most 32 and at most Rp)
int tc_nt(int Rp, int tile)
{
    int nt = (tile >= 8 ? tile : 32) / 8;
    if (nt > 4) nt = 4;
    if (nt * 8 > Rp) nt = Rp / 8;
    return nt;
}

int tc_blocks_per_sm(int Rp, int threads, int tile)
{
    switch (tc_nt(Rp, tile)) {
    case 1: return tc_fit<1>(threads);
    case 2: return tc_fit<2>(threads);
    case 4: return tc_fit<4>(threads);
    }
    return 0;
}

cudaError_t launch_tc_step(const StepArgs &a, int Rp, int tile, int blocks, int threads, bool functionals,
                           cudaStream_t s)
{
    cudaError_t e;
    if (functionals) {
        if (a.det && a.n_patch > 0) {
            tc_det_kernel<<<a.n_patch, kMaxRhs, 0, s>>>(a, Rp);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // 8 warps per block: a multiple of Rp blocks keeps each warp on one rhs
        const int nb = ((sms * 4 + Rp - 1) / Rp) * Rp;
        tc_ledger_kernel<<<nb, 256, 0, s>>>(a, Rp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    switch (tc_nt(Rp, tile)) {
    case 1: tc_step_kernel<1><<<blocks, threads, 0, s>>>(a, Rp); break;
    case 2: tc_step_kernel<2><<<blocks, threads, 0, s>>>(a, Rp); break;
    case 4: tc_step_kernel<4><<<blocks, threads, 0, s>>>(a, Rp); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_tc_to_canonical(const void *x, int64_t V, int Rp, int r, double *out, cudaStream_t s)
{
    const int th = 256;
    tc_to_canonical_kernel<<<unsigned((V * kDirs + th - 1) / th), th, 0, s>>>(static_cast<const float *>(x), V, Rp,
                                                                               r, out);
    return cudaGetLastError();
}

cudaError_t launch_tc_from_canonical(const double *in, int64_t V, int Rp, int r, void *x, cudaStream_t s)
{
    const int th = 256;
    tc_from_canonical_kernel<<<unsigned((V * kDirs + th - 1) / th), th, 0, s>>>(in, V, Rp, r,
                                                                                 static_cast<float *>(x));
    return cudaGetLastError();
}

cudaError_t launch_tc_sum(const void *x, int64_t V, int Rp, int r, double *out, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    tc_sum_kernel<<<sms * 2, 256, 0, s>>>(static_cast<const float *>(x), V, Rp, r, out);
    return cudaGetLastError();
}

}  // namespace drts
