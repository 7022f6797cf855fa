// Batched DRTS step X(t+1) = A X(t) + S(t) for R right-hand sides that
// share one assembled A (the paper notes that only the source term changes
// between such runs, Section 6).  One pass over A serves RT right-hand sides
// at a time: every nonzero's value and code are loaded once and used for RT
// multiply-adds against X[r0 .. r0+RT)[column].
//
// State layout: right-hand sides in groups of four, each group state-major
// with the group's four values of a state side by side:
//   X[((r/4) * rhs_stride + n*V + v) * 4 + r%4].
// For one code the 32 lanes of a slice (32 consecutive voxels) read 32
// consecutive 16-byte vectors, i.e. one coalesced 512-byte request serves
// four right-hand sides with a single load instruction per lane.
//
// Accumulation: products are chained with FMA and the chain is added to a
// Kahan-compensated accumulator (plain FP32 sums of ~200 positive terms
// drift the solution by ~1e-7 per step).  With 4 right-hand sides per pass
// a chain covers four groups (16 products), which saves instructions;
// wider tiles add every group.
//
// The detector readout (Eq. 27) and the FP64 ledger of X(t) come from two
// small kernels launched before the product: one block per detector patch
// (a deterministic sum, no atomics) and a reduction per right-hand side.
#include <cuda_runtime.h>

#include <type_traits>

#include "drts_device.cuh"
#include "drts_kernel_common.cuh"

namespace drts {
namespace {

// value of source entry e at this step
__device__ __forceinline__ double source_value(const StepArgs &a, const SourceEntry &e)
{
    if (a.step_scale) return e.w * a.step_scale[e.rhs];
    const SourceProfile &p = a.prof[e.prof];
    if (a.t >= p.t0 && a.t < p.t0 + p.n_t) return e.w * a.prof_vals[p.off + (a.t - p.t0)];
    return 0.0;
}

// first source entry whose slice is >= q (entries are sorted by slice)
__device__ __forceinline__ int first_entry(const SourceEntry *src, int n, int64_t q)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (src[mid].slice < q) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <class AT>
struct KahanAcc {
    AT s = 0, c = 0;
    __device__ __forceinline__ void add(AT v)
    {
        const AT y = v - c;
        const AT t = s + y;
        c = (t - s) - y;
        s = t;
    }
};
template <>
struct KahanAcc<double> {
    double s = 0, c = 0;
    __device__ __forceinline__ void add(double v) { s += v; }
};

// the four values of state o in a group of right-hand sides
__device__ __forceinline__ void load_rhs4(const float *g, int32_t o, float out[4])
{
    const float4 t = __ldg(reinterpret_cast<const float4 *>(g) + o);
    out[0] = t.x; out[1] = t.y; out[2] = t.z; out[3] = t.w;
}
__device__ __forceinline__ void load_rhs4(const float *g, int64_t o, float out[4])
{
    const float4 t = __ldg(reinterpret_cast<const float4 *>(g) + o);
    out[0] = t.x; out[1] = t.y; out[2] = t.z; out[3] = t.w;
}
__device__ __forceinline__ void load_rhs4(const double *g, int64_t o, double out[4])
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(g) + 2 * o);
    const double2 b = __ldg(reinterpret_cast<const double2 *>(g) + 2 * o + 1);
    out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}
__device__ __forceinline__ void store_rhs4(float *g, int64_t o, const float v[4])
{
    reinterpret_cast<float4 *>(g)[o] = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store_rhs4(double *g, int64_t o, const double v[4])
{
    reinterpret_cast<double2 *>(g)[2 * o] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(g)[2 * o + 1] = make_double2(v[2], v[3]);
}

// ORDER 0: warps stride over slices (consecutive warps take consecutive
// slices of the whole matrix).  ORDER 1: block-major - the CTA owns voxel
// blocks b = blockIdx.x + k * gridDim.x and its warps share out the 26 slices
// (directions m) of those blocks in turn, so the x neighbourhood of one voxel
// block (read by all 26 of its slices) is gathered by warps of the same SM
// while it is still in L1.
// The FP32 8-per-pass instance is held to 64 registers so that four
// 256-thread CTAs fit an SM (32 warps to hide the gathers' L2 latency; at
// 66 registers only three fit, and the step ran ~13 % slower).
template <class VT, class XT, class AT, int RT, int ORDER>
__global__ void __launch_bounds__(256, (RT == 8 && sizeof(XT) == 4) ? 4 : 1) spmm_kernel(StepArgs a, int r0)
{
    __shared__ int32_t s_delta[kCodes];
    const int64_t V = a.V;
    for (int c = threadIdx.x; c < kCodes; c += blockDim.x) {
        const int d = c / kDirs, n = c % kDirs;
        s_delta[c] = int32_t(n * V + (int64_t(d / 9 - 1) * a.ny + (d / 3 % 3 - 1)) * a.nx + (d % 3 - 1));
    }
    __syncthreads();
    const int64_t S = a.rhs_stride;
    const int nr = a.R - r0 < RT ? a.R - r0 : RT;   // right-hand sides in this tile
    constexpr int NG = RT / 4;                       // groups of four per tile
    const int ngr = (nr + 3) >> 2;                   // groups holding live right-hand sides
    const XT *__restrict__ x = static_cast<const XT *>(a.x) + int64_t(r0 >> 2) * 4 * S;
    XT *__restrict__ y = static_cast<XT *>(a.y) + int64_t(r0 >> 2) * 4 * S;
    const VT *__restrict__ vals = static_cast<const VT *>(a.A.vals);
    const uint16_t *__restrict__ codes = a.A.codes;
    const int lane = threadIdx.x & 31;
    int64_t first, count, stride;
    if (ORDER == 0) {
        first = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
        stride = (int64_t(gridDim.x) * blockDim.x) >> 5;
        count = a.A.n_slices;
    } else {
        // items i = (k, m) of this CTA's blocks, k-major; warp w takes w, w + nw, ...
        const int64_t nb = a.A.n_slices / kDirs;
        const int64_t mine = blockIdx.x < nb ? (nb - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
        first = threadIdx.x >> 5;
        stride = blockDim.x >> 5;
        count = mine * kDirs;
    }

    for (int64_t it = first; it < count; it += stride) {
        int64_t q;
        if (ORDER == 0) {
            q = it;
        } else {
            const int64_t k = it / kDirs;
            q = (int64_t(blockIdx.x) + k * gridDim.x) * kDirs + (it - k * kDirs);
        }
        const int64_t b = q / kDirs;
        const int m = int(q - b * kDirs);
        const int64_t v = b * kSlice + lane;
        const int len4 = a.A.slice_len4[q];
        const int64_t base = a.A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup;
        KahanAcc<AT> acc[RT];
        AT wn[4];
        int cn[4];
        if (len4 > 0) {
            load4(vals + base, wn);
            load_codes(codes + base, cn);
        }
        // state indices fit 32 bits (fewer than 2^31 states); 32-bit offsets
        // save address arithmetic for narrow FP32 tiles, the others keep
        // 64-bit ones (fewer registers for wide tiles; FP64 vectors index
        // twice the offset)
        using OT = typename std::conditional<(RT <= 4 && sizeof(XT) == 4), int32_t, int64_t>::type;
        const OT v32 = OT(v);
        // products of H groups per compensated addition: four while the tile
        // is narrow (fewer additions); one for wider tiles, where longer
        // chains measured slower (RT 8: 2.5x against 3.1x per simulation)
        constexpr int H = RT <= 4 ? 4 : 1;
        for (int g0 = 0; g0 < len4; g0 += H) {
            AT p[RT];
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const int g = g0 + h;
                if (g >= len4) break;
                AT w[4];
                int c[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) { w[j] = wn[j]; c[j] = cn[j]; }
                if (g + 1 < len4) {
                    const int64_t idx = base + int64_t(g + 1) * (kSlice * kGroup);
                    load4(vals + idx, wn);
                    load_codes(codes + idx, cn);
                }
                const OT o0 = v32 + s_delta[c[0]], o1 = v32 + s_delta[c[1]];
                const OT o2 = v32 + s_delta[c[2]], o3 = v32 + s_delta[c[3]];
#pragma unroll
                for (int gi = 0; gi < NG; ++gi) {
                    if (gi < ngr) {
                        const XT *xg = x + int64_t(gi) * 4 * S;
                        XT x0[4], x1[4], x2[4], x3[4];
                        load_rhs4(xg, o0, x0);
                        load_rhs4(xg, o1, x1);
                        load_rhs4(xg, o2, x2);
                        load_rhs4(xg, o3, x3);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int r = gi * 4 + k;
                            AT q = h ? fma(w[0], AT(x0[k]), p[r]) : w[0] * AT(x0[k]);
                            q = fma(w[1], AT(x1[k]), q);
                            q = fma(w[2], AT(x2[k]), q);
                            q = fma(w[3], AT(x3[k]), q);
                            if constexpr (H == 1) acc[r].add(q);
                            else p[r] = q;
                        }
                    }
                }
            }
            if constexpr (H > 1) {
#pragma unroll
                for (int r = 0; r < RT; ++r)
                    if ((r >> 2) < ngr) acc[r].add(p[r]);
            }
        }
        if (v >= V) continue;
        const AT sc = a.A.row_scale ? AT(a.A.row_scale[q * kSlice + lane]) : AT(1);
        AT out[RT];
#pragma unroll
        for (int r = 0; r < RT; ++r) out[r] = acc[r].s * sc;
        if (a.n_src > 0) {
            for (int e = first_entry(a.src, a.n_src, q); e < a.n_src && a.src[e].slice == q; ++e) {
                const SourceEntry se = a.src[e];
                if (se.lane != lane) continue;
                const int rr = se.rhs - r0;
                const AT val = AT(source_value(a, se));
#pragma unroll
                for (int r = 0; r < RT; ++r)
                    if (r == rr) out[r] += val;
            }
        }
        const int64_t row = int64_t(m) * V + v;
#pragma unroll
        for (int gi = 0; gi < NG; ++gi)
            if (gi < ngr) {
                XT o4[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) o4[k] = XT(out[gi * 4 + k]);
                store_rhs4(y + int64_t(gi) * 4 * S, row, o4);
            }
    }
}

// ORDER 2: the x halo of one voxel block in shared memory.  A CTA of 26
// warps owns voxel blocks b = blockIdx.x + k * gridDim.x; for each tile of RT
// right-hand sides it first stages every x value the block's 26 x 32 rows
// can read - nine row ranges (dy, dz) of 34 voxels (the 32 of the block and
// one on each side), 26 directions, RT right-hand sides, stored
// [range][n][voxel][r] - then warp m computes slice (b, m) from shared
// memory: one 16-byte load gives the RT values of a code.  Every x value is
// then read from L2 once per block instead of once per row, and the gathers
// no longer miss.  RT = 16 bytes / sizeof(XT): 4 FP32 or 2 FP64 values
// (127,296 bytes of halo).
constexpr int kHaloRanges = 9, kHaloVox = kSlice + 2;
constexpr int kHaloThreads = kDirs * 32;

template <class XT>
struct HaloRT {
    static constexpr int value = 16 / int(sizeof(XT));
};

__device__ __forceinline__ void load_rt(const float *p, float o[4])
{
    const float4 t = *reinterpret_cast<const float4 *>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void load_rt(const double *p, double o[2])
{
    const double2 t = *reinterpret_cast<const double2 *>(p);
    o[0] = t.x; o[1] = t.y;
}

template <class XT>
constexpr size_t halo_smem_bytes()
{
    return size_t(kHaloRanges) * kDirs * kHaloVox * HaloRT<XT>::value * sizeof(XT) + kCodes * sizeof(int32_t);
}

template <class VT, class XT, class AT>
__global__ void __launch_bounds__(kHaloThreads, 1) spmm_halo_kernel(StepArgs a)
{
    constexpr int RT = HaloRT<XT>::value;
    extern __shared__ __align__(16) unsigned char halo_raw[];
    XT *xs = reinterpret_cast<XT *>(halo_raw);
    int32_t *s_off = reinterpret_cast<int32_t *>(xs + kHaloRanges * kDirs * kHaloVox * RT);
    for (int c = threadIdx.x; c < kCodes; c += blockDim.x) {
        const int d = c / kDirs, n = c % kDirs;
        const int rr = (d / 9) * 3 + (d / 3 % 3);            // (dz + 1) * 3 + (dy + 1)
        s_off[c] = ((rr * kDirs + n) * kHaloVox + d % 3) * RT;  // voxel slot lane + dx + 1
    }
    const int64_t V = a.V;
    const int64_t S = a.rhs_stride;
    const XT *__restrict__ x = static_cast<const XT *>(a.x);
    XT *__restrict__ y = static_cast<XT *>(a.y);
    const VT *__restrict__ vals = static_cast<const VT *>(a.A.vals);
    const uint16_t *__restrict__ codes = a.A.codes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int64_t n_vb = a.A.n_slices / kDirs;
    constexpr int kHaloElems = kHaloRanges * kDirs * kHaloVox;
    for (int64_t b = blockIdx.x; b < n_vb; b += gridDim.x) {
        const int64_t v0 = b * kSlice;
        for (int r0 = 0; r0 < a.R; r0 += RT) {
            const int nr = a.R - r0 < RT ? a.R - r0 : RT;
            __syncthreads();                 // the previous tile's readers are done
            for (int i = threadIdx.x; i < kHaloElems * RT; i += blockDim.x) {
                const int p = i % kHaloVox;
                int rest = i / kHaloVox;
                const int n = rest % kDirs;
                rest /= kDirs;
                const int rr = rest % kHaloRanges;
                const int r = rest / kHaloRanges;
                const int64_t g = v0 + (int64_t(rr / 3 - 1) * a.ny + (rr % 3 - 1)) * a.nx - 1 + p;
                XT val = XT(0);
                const int ra = r0 + r;
                if (r < nr && g >= 0 && g < V) val = x[(int64_t(ra >> 2) * S + int64_t(n) * V + g) * 4 + (ra & 3)];
                xs[((rr * kDirs + n) * kHaloVox + p) * RT + r] = val;
            }
            __syncthreads();
            for (int m = warp; m < kDirs; m += nwarps) {
                const int64_t q = b * kDirs + m;
                const int64_t v = v0 + lane;
                const int len4 = a.A.slice_len4[q];
                const int64_t base = a.A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup;
                KahanAcc<AT> acc[RT];
                AT wn[4];
                int cn[4];
                if (len4 > 0) {
                    load4(vals + base, wn);
                    load_codes(codes + base, cn);
                }
                for (int g = 0; g < len4; ++g) {
                    AT w[4];
                    int c[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) { w[j] = wn[j]; c[j] = cn[j]; }
                    if (g + 1 < len4) {
                        const int64_t idx = base + int64_t(g + 1) * (kSlice * kGroup);
                        load4(vals + idx, wn);
                        load_codes(codes + idx, cn);
                    }
                    XT xv[4][RT];
#pragma unroll
                    for (int j = 0; j < 4; ++j) load_rt(xs + s_off[c[j]] + lane * RT, xv[j]);
#pragma unroll
                    for (int r = 0; r < RT; ++r) {
                        AT p = w[0] * AT(xv[0][r]);
                        p = fma(w[1], AT(xv[1][r]), p);
                        p = fma(w[2], AT(xv[2][r]), p);
                        p = fma(w[3], AT(xv[3][r]), p);
                        acc[r].add(p);
                    }
                }
                if (v >= V) continue;
                const AT sc = a.A.row_scale ? AT(a.A.row_scale[q * kSlice + lane]) : AT(1);
                AT out[RT];
#pragma unroll
                for (int r = 0; r < RT; ++r) out[r] = acc[r].s * sc;
                if (a.n_src > 0) {
                    for (int e = first_entry(a.src, a.n_src, q); e < a.n_src && a.src[e].slice == q; ++e) {
                        const SourceEntry se = a.src[e];
                        if (se.lane != lane) continue;
                        const int rr = se.rhs - r0;
                        const AT val = AT(source_value(a, se));
#pragma unroll
                        for (int r = 0; r < RT; ++r)
                            if (r == rr) out[r] += val;
                    }
                }
                const int64_t row = int64_t(m) * V + v;
#pragma unroll
                for (int r = 0; r < RT; ++r)
                    if (r < nr) {
                        const int ra = r0 + r;
                        y[(int64_t(ra >> 2) * S + row) * 4 + (ra & 3)] = XT(out[r]);
                    }
            }
        }
    }
}

template <class VT, class XT, class AT>
int halo_blocks_per_sm()
{
    // the shared-memory opt-in is a per-device function attribute: set it
    // once on every device the kernel is used on
    static bool attr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 0;
    }
    if (!attr[dev]) {
        if (cudaFuncSetAttribute(spmm_halo_kernel<VT, XT, AT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(halo_smem_bytes<XT>())) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        attr[dev] = true;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, spmm_halo_kernel<VT, XT, AT>, kHaloThreads,
                                                      halo_smem_bytes<XT>()) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <class VT, class XT, class AT>
cudaError_t launch_halo(const StepArgs &a, cudaStream_t s)
{
    const int per = halo_blocks_per_sm<VT, XT, AT>();
    if (per < 1) return cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    spmm_halo_kernel<VT, XT, AT><<<sms * per, kHaloThreads, halo_smem_bytes<XT>(), s>>>(a);
    return cudaGetLastError();
}

// Absorbed and exited mass of X(t) per right-hand side (FP64 ledger) and the
// injected mass of this step.  blockIdx.y is the right-hand side.
template <class XT>
__global__ void __launch_bounds__(256) ledger_kernel(StepArgs a)
{
    __shared__ double red[2];
    if (threadIdx.x < 2) red[threadIdx.x] = 0.0;
    __syncthreads();
    const int r = blockIdx.y;
    const XT *x = static_cast<const XT *>(a.x) + int64_t(r >> 2) * 4 * a.rhs_stride + (r & 3);
    const int64_t total = a.V * kDirs;
    float ab = 0.0f, ex = 0.0f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const float xs = float(x[i * 4]);
        if (xs == 0.0f) continue;
        const int d = int(i / a.V);
        const int64_t v = i - int64_t(d) * a.V;
        const int k = a.cls[v];
        ab += float(a.tab.absorb_dir ? a.tab.absorb_dir[k * kDirs + d] : a.tab.absorb[k]) * xs;
        const int xx = int(v % a.nx), yy = int(v / a.nx % a.ny), zz = int(v / (int64_t(a.nx) * a.ny));
        const int mask = (zz == 0 ? 0 : (zz == a.nz - 1 ? 2 : 1)) * 9 +
                         (yy == 0 ? 0 : (yy == a.ny - 1 ? 2 : 1)) * 3 + (xx == 0 ? 0 : (xx == a.nx - 1 ? 2 : 1));
        if (mask != 13) ex += float(a.tab.exit_total[(k * 27 + mask) * kDirs + d]) * xs;
    }
    const float abw = warp_sum(ab), exw = warp_sum(ex);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&red[0], double(abw));
        atomicAdd(&red[1], double(exw));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (red[0] != 0.0) atomicAdd(&a.ledger[4 * r + 2], red[0]);
        if (red[1] != 0.0) atomicAdd(&a.ledger[4 * r + 3], red[1]);
        if (blockIdx.x == 0)
            for (int e = 0; e < a.n_src; ++e)
                if (a.src[e].rhs == r) {
                    const double val = source_value(a, a.src[e]);
                    if (val != 0.0) atomicAdd(&a.ledger[4 * r + 1], val);
                }
    }
}

// Detector readout of X(t): one block per patch, one thread per right-hand
// side; each thread sums its patch in a fixed order (no atomics).
template <class XT>
__global__ void det_kernel(StepArgs a)
{
    const int p = blockIdx.x;
    const int r = threadIdx.x;
    if (r >= a.R) return;
    const int fa = a.det_face >> 1, high = a.det_face & 1;
    const int N[3] = {a.nx, a.ny, a.nz};
    const int ua = fa == 0 ? 1 : 0, va = fa == 2 ? 1 : 2;
    const int pu = p % a.det_nu, pv = p / a.det_nu;
    const int Nu = N[ua], Nv = N[va];
    const int u0 = (pu * Nu + a.det_nu - 1) / a.det_nu, u1 = ((pu + 1) * Nu + a.det_nu - 1) / a.det_nu;
    const int v0 = (pv * Nv + a.det_nv - 1) / a.det_nv, v1 = ((pv + 1) * Nv + a.det_nv - 1) / a.det_nv;
    const XT *x = static_cast<const XT *>(a.x) + int64_t(r >> 2) * 4 * a.rhs_stride + (r & 3);
    double sum = 0.0;
    for (int cv = v0; cv < v1; ++cv)
        for (int cu = u0; cu < u1; ++cu) {
            int c[3];
            c[fa] = high ? N[fa] - 1 : 0;
            c[ua] = cu;
            c[va] = cv;
            const int64_t v = (int64_t(c[2]) * a.ny + c[1]) * a.nx + c[0];
            const int k = a.cls[v];
            const int mask = (c[2] == 0 ? 0 : (c[2] == a.nz - 1 ? 2 : 1)) * 9 +
                             (c[1] == 0 ? 0 : (c[1] == a.ny - 1 ? 2 : 1)) * 3 +
                             (c[0] == 0 ? 0 : (c[0] == a.nx - 1 ? 2 : 1));
            for (int d = 0; d < kDirs; ++d) {
                const double ed = a.tab.exit_det[(k * 27 + mask) * kDirs + d];
                if (ed > 0.0) sum += ed * double(x[(int64_t(d) * a.V + v) * 4]);
            }
        }
    a.det[r * a.det_stride_r + p] = sum;
}

template <class VT, class XT, class AT>
struct SpmmLaunch {
    template <int RT, int ORDER>
    static int fit(int threads)
    {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, spmm_kernel<VT, XT, AT, RT, ORDER>, threads, 0) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return n;
    }
    template <int ORDER>
    static int per_sm_order(int rt, int threads)
    {
        switch (rt) {
        case 4: return fit<4, ORDER>(threads);
        case 8: return fit<8, ORDER>(threads);
        case 16: return fit<16, ORDER>(threads);
        case 32: return fit<32, ORDER>(threads);
        }
        return 0;
    }
    static int per_sm(int rt, int threads, int order)
    {
        if (order == 2) return halo_blocks_per_sm<VT, XT, AT>();
        return order == 0 ? per_sm_order<0>(rt, threads) : per_sm_order<1>(rt, threads);
    }
    template <int ORDER>
    static cudaError_t launch_order(int rt, const StepArgs &a, int r0, int blocks, int threads, cudaStream_t s)
    {
        switch (rt) {
        case 4: spmm_kernel<VT, XT, AT, 4, ORDER><<<blocks, threads, 0, s>>>(a, r0); break;
        case 8: spmm_kernel<VT, XT, AT, 8, ORDER><<<blocks, threads, 0, s>>>(a, r0); break;
        case 16: spmm_kernel<VT, XT, AT, 16, ORDER><<<blocks, threads, 0, s>>>(a, r0); break;
        case 32: spmm_kernel<VT, XT, AT, 32, ORDER><<<blocks, threads, 0, s>>>(a, r0); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    static cudaError_t launch(int rt, int order, const StepArgs &a, int r0, int blocks, int threads,
                              cudaStream_t s)
    {
        return order == 0 ? launch_order<0>(rt, a, r0, blocks, threads, s)
                          : launch_order<1>(rt, a, r0, blocks, threads, s);
    }
};

}  // namespace

int batched_blocks_per_sm(int precision, int rhs_tile, int threads, int order)
{
    if (precision == DRTS_FP64) return SpmmLaunch<double, double, double>::per_sm(rhs_tile, threads, order);
    if (precision == DRTS_FP32) return SpmmLaunch<float, float, float>::per_sm(rhs_tile, threads, order);
    return SpmmLaunch<__half, float, float>::per_sm(rhs_tile, threads, order);
}

cudaError_t launch_batched_step(const StepArgs &a, int n_rhs, int rhs_tile, int order, int blocks, int threads,
                                bool functionals, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    const bool f64 = a.A.precision == DRTS_FP64;
    if (functionals) {
        if (a.det && a.n_patch > 0) {
            if (f64) det_kernel<double><<<a.n_patch, kMaxRhs, 0, s>>>(a);
            else det_kernel<float><<<a.n_patch, kMaxRhs, 0, s>>>(a);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const dim3 grid(unsigned((sms * 4 + n_rhs - 1) / n_rhs), unsigned(n_rhs));
        if (f64) ledger_kernel<double><<<grid, 256, 0, s>>>(a);
        else ledger_kernel<float><<<grid, 256, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (order == 2) {           // one launch: the kernel loops over the right-hand-side tiles
        if (a.A.precision == DRTS_FP64) return launch_halo<double, double, double>(a, s);
        if (a.A.precision == DRTS_FP32) return launch_halo<float, float, float>(a, s);
        return launch_halo<__half, float, float>(a, s);
    }
    for (int r0 = 0; r0 < n_rhs; r0 += rhs_tile) {
        if (a.A.precision == DRTS_FP64)
            e = SpmmLaunch<double, double, double>::launch(rhs_tile, order, a, r0, blocks, threads, s);
        else if (a.A.precision == DRTS_FP32)
            e = SpmmLaunch<float, float, float>::launch(rhs_tile, order, a, r0, blocks, threads, s);
        else
            e = SpmmLaunch<__half, float, float>::launch(rhs_tile, order, a, r0, blocks, threads, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace drts
