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
#include "drts_functionals.cuh"
#include "drts_kernel_common.cuh"

namespace drts {
namespace {

// Compensated accumulator: FP32 rows sum ~200 products, and plain FP32
// accumulation drifts the solution by a few 1e-6 per 1000 steps.  Products are
// summed pairwise inside a group of four and the group sums are added with
// Kahan compensation.  FP64 rows accumulate plainly.
template <class AT>
struct Acc {
    AT s = 0, c = 0;
    __device__ __forceinline__ void add(AT v)
    {
        const AT y = v - c;
        const AT t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ AT value() const { return s; }
};
template <>
struct Acc<double> {
    double s = 0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};

// Group data held in registers: four values (widened to AT) and four codes.
template <class AT>
struct Group {
    AT w[4];
    int c[4];
};

template <class VT, class AT>
__device__ __forceinline__ void load_group(const VT *vals, const uint16_t *codes, int64_t idx, Group<AT> &g)
{
    load4(vals + idx, g.w);
    load_codes(codes + idx, g.c);
}

// A group as loaded: the raw 16-byte / 8-byte words, unpacked only when
// used, so a prefetched group costs 6 registers (FP32), 4 (FP16) or 10 (FP64).
template <class VT>
struct RawGroup;
template <>
struct RawGroup<float> {
    float4 w;
    uint2 c;
};
template <>
struct RawGroup<__half> {
    uint2 w;
    uint2 c;
};
template <>
struct RawGroup<double> {
    double2 w0, w1;
    uint2 c;
};

__device__ __forceinline__ void load_raw(const float *vals, const uint16_t *codes, int64_t idx, RawGroup<float> &g)
{
    g.w = __ldcs(reinterpret_cast<const float4 *>(vals + idx));
    g.c = __ldcs(reinterpret_cast<const uint2 *>(codes + idx));
}
__device__ __forceinline__ void load_raw(const __half *vals, const uint16_t *codes, int64_t idx,
                                         RawGroup<__half> &g)
{
    g.w = __ldcs(reinterpret_cast<const uint2 *>(vals + idx));
    g.c = __ldcs(reinterpret_cast<const uint2 *>(codes + idx));
}
__device__ __forceinline__ void load_raw(const double *vals, const uint16_t *codes, int64_t idx,
                                         RawGroup<double> &g)
{
    g.w0 = __ldcs(reinterpret_cast<const double2 *>(vals + idx));
    g.w1 = __ldcs(reinterpret_cast<const double2 *>(vals + idx) + 1);
    g.c = __ldcs(reinterpret_cast<const uint2 *>(codes + idx));
}

__device__ __forceinline__ void unpack(const RawGroup<float> &g, float w[4])
{
    w[0] = g.w.x; w[1] = g.w.y; w[2] = g.w.z; w[3] = g.w.w;
}
__device__ __forceinline__ void unpack(const RawGroup<__half> &g, float w[4])
{
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&g.w.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&g.w.y));
    w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
}
__device__ __forceinline__ void unpack(const RawGroup<double> &g, double w[4])
{
    w[0] = g.w0.x; w[1] = g.w0.y; w[2] = g.w1.x; w[3] = g.w1.y;
}

// State loads: through the read-only cache when x is not written during the
// kernel; coherent (L2) loads in the persistent kernel, which writes the
// buffer it reads in the next step.  (Ordinary L1-cached loads after the
// grid barrier measured slower there: 118 vs 97 us per step at 16^3 FP64,
// 61.5 vs 44.7 ms at 192^3 FP16.)
template <bool COHERENT, class XT>
__device__ __forceinline__ XT load_x(const XT *p)
{
    if constexpr (COHERENT) return __ldcg(p);
    else return __ldg(p);
}

// Dot product of one row with x, streaming the row's groups with D groups
// prefetched ahead so that D matrix loads per lane are in flight while the
// current group's x gathers run.
template <class VT, class XT, class AT, int D, bool COHERENT = false>
__device__ __forceinline__ AT row_dot(const VT *__restrict__ vals, const uint16_t *__restrict__ codes,
                                      int64_t base, int len4, const XT *__restrict__ x, int64_t v,
                                      const int32_t *s_delta)
{
    RawGroup<VT> buf[D];
#pragma unroll
    for (int s = 0; s < D; ++s)
        if (s < len4) load_raw(vals, codes, base + int64_t(s) * (kSlice * kGroup), buf[s]);
    Acc<AT> acc;
    for (int g0 = 0; g0 < len4; g0 += D) {
#pragma unroll
        for (int s = 0; s < D; ++s) {
            const int g = g0 + s;
            if (g < len4) {
                const RawGroup<VT> cur = buf[s];
                if (g + D < len4) load_raw(vals, codes, base + int64_t(g + D) * (kSlice * kGroup), buf[s]);
                AT w[4];
                unpack(cur, w);
                const int c0 = int(cur.c.x & 0xffffu), c1 = int(cur.c.x >> 16);
                const int c2 = int(cur.c.y & 0xffffu), c3 = int(cur.c.y >> 16);
                const AT p0 = w[0] * AT(load_x<COHERENT>(x + (v + s_delta[c0])));
                const AT p1 = w[1] * AT(load_x<COHERENT>(x + (v + s_delta[c1])));
                const AT p2 = w[2] * AT(load_x<COHERENT>(x + (v + s_delta[c2])));
                const AT p3 = w[3] * AT(load_x<COHERENT>(x + (v + s_delta[c3])));
                acc.add((p0 + p1) + (p2 + p3));
            }
        }
    }
    return acc.value();
}

// Shared per-block data of a step: the code -> state-offset table, the
// block's ledger partials and this step's source values.
struct StepShared {
    int32_t delta[kCodes];
    double ledger[2];
    SourceEntry src[kMaxSrc];
    double src_val[kMaxSrc];
};

__device__ __forceinline__ void step_delta(const StepArgs &a, StepShared &sh)
{
    for (int c = threadIdx.x; c < kCodes; c += blockDim.x) {
        const int d = c / kDirs, n = c % kDirs;
        sh.delta[c] = int32_t(n * a.V + (int64_t(d / 9 - 1) * a.ny + (d / 3 % 3 - 1)) * a.nx + (d % 3 - 1));
    }
}

// this step's source values and a zeroed block ledger (ends with a barrier)
__device__ __forceinline__ void step_sources(const StepArgs &a, StepShared &sh)
{
    if (threadIdx.x < 2) sh.ledger[threadIdx.x] = 0.0;
    for (int e = threadIdx.x; e < a.n_src; e += blockDim.x) {
        sh.src[e] = a.src[e];
        const SourceProfile &p = a.prof[a.src[e].prof];
        double val = 0.0;
        if (a.step_scale) val = a.src[e].w * a.step_scale[a.src[e].rhs];
        else if (a.t >= p.t0 && a.t < p.t0 + p.n_t) val = a.src[e].w * a.prof_vals[p.off + (a.t - p.t0)];
        sh.src_val[e] = val;
    }
    __syncthreads();
}

__device__ __forceinline__ void step_prologue(const StepArgs &a, StepShared &sh)
{
    step_delta(a, sh);
    step_sources(a, sh);
}

// Finish row (voxel v, direction m) of slice q: row scale, source term, store,
// and the column functionals of x(t) for the same state (Eq. 27, ledger).
template <class XT, class AT, bool COHERENT = false>
__device__ __forceinline__ void row_epilogue(const StepArgs &a, const StepShared &sh, int64_t q, int lane,
                                             int64_t v, int m, AT acc, AT &ab_lane, AT &ex_lane)
{
    if (a.A.row_scale) acc *= AT(a.A.row_scale[q * kSlice + lane]);
    if (v >= a.V) return;
    const XT *x = static_cast<const XT *>(a.x);
    XT *y = static_cast<XT *>(a.y);
    const int64_t row = int64_t(m) * a.V + v;
    for (int e = 0; e < a.n_src; ++e)
        if (sh.src[e].slice == q && sh.src[e].lane == lane) acc += AT(sh.src_val[e]);
    y[row] = XT(acc);
    const AT xs = AT(COHERENT ? __ldcg(x + row) : x[row]);
    const int k = a.cls[v];
    ab_lane += AT(a.tab.absorb_dir ? a.tab.absorb_dir[k * kDirs + m] : a.tab.absorb[k]) * xs;
    const int nxy = a.nx * a.ny;
    const int xx = int(v % a.nx), yy = int(v / a.nx % a.ny), zz = int(v / nxy);
    const int bx = xx == 0 ? 0 : (xx == a.nx - 1 ? 2 : 1);
    const int by = yy == 0 ? 0 : (yy == a.ny - 1 ? 2 : 1);
    const int bz = zz == 0 ? 0 : (zz == a.nz - 1 ? 2 : 1);
    const int mask = bz * 9 + by * 3 + bx;
    if (mask == 13) return;
    const int ti = (k * 27 + mask) * kDirs + m;
    ex_lane += AT(a.tab.exit_total[ti]) * xs;
    const double ed = a.tab.exit_det[ti];
    if (ed > 0.0 && a.det) {
        // patch coordinates (u, v) = the two other axes in x, y, z order
        const int fa = a.det_face >> 1;
        const int cu = fa == 0 ? yy : xx, nu = fa == 0 ? a.ny : a.nx;
        const int cv = fa == 2 ? yy : zz, nv = fa == 2 ? a.ny : a.nz;
        const int p = int(int64_t(cv) * a.det_nv / nv) * a.det_nu + int(int64_t(cu) * a.det_nu / nu);
        atomicAdd(a.det + p, ed * double(xs));
    }
}

template <class AT>
__device__ __forceinline__ void step_finish(const StepArgs &a, StepShared &sh, AT ab_lane, AT ex_lane)
{
    const AT ab_w = warp_sum(ab_lane), ex_w = warp_sum(ex_lane);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sh.ledger[0], double(ab_w));
        atomicAdd(&sh.ledger[1], double(ex_w));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sh.ledger[0] != 0.0) atomicAdd(&a.ledger[2], sh.ledger[0]);
        if (sh.ledger[1] != 0.0) atomicAdd(&a.ledger[3], sh.ledger[1]);
        if (blockIdx.x == 0) {          // injected mass, once per step
            double inj = 0.0;
            for (int e = 0; e < a.n_src; ++e) inj += sh.src_val[e];
            if (inj != 0.0) atomicAdd(&a.ledger[1], inj);
        }
    }
}

// Row dot product with both streams software-pipelined: the matrix group
// two ahead is loading and the x values of the next group are being gathered
// while the current group's products accumulate, so neither the HBM latency
// of the matrix nor the L1/L2 latency of the gathers sits on the critical path.
template <class VT, class XT, class AT>
__device__ __forceinline__ AT row_dot_pipelined(const VT *__restrict__ vals, const uint16_t *__restrict__ codes,
                                                int64_t base, int len4, const XT *__restrict__ x, int64_t v,
                                                const int32_t *s_delta)
{
    constexpr int64_t kStride = kSlice * kGroup;
    Group<AT> g1, g2;                  // matrix groups g+1 and g+2
    AT w0[4], x0[4];                   // current group: values and gathered x
    Acc<AT> acc;
    if (len4 <= 0) return acc.value();
    {
        Group<AT> g0;
        load_group(vals, codes, base, g0);
        if (len4 > 1) load_group(vals, codes, base + kStride, g1);
        if (len4 > 2) load_group(vals, codes, base + 2 * kStride, g2);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            w0[j] = g0.w[j];
            x0[j] = AT(__ldg(x + (v + s_delta[g0.c[j]])));
        }
    }
    for (int g = 0; g < len4; ++g) {
        AT w1[4], x1[4];
        if (g + 1 < len4) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                w1[j] = g1.w[j];
                x1[j] = AT(__ldg(x + (v + s_delta[g1.c[j]])));
            }
            g1 = g2;
            if (g + 3 < len4) load_group(vals, codes, base + int64_t(g + 3) * kStride, g2);
        }
        acc.add((w0[0] * x0[0] + w0[1] * x0[1]) + (w0[2] * x0[2] + w0[3] * x0[3]));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            w0[j] = w1[j];
            x0[j] = x1[j];
        }
    }
    return acc.value();
}

// Variant 9: registers path with both streams pipelined.
template <class VT, class XT, class AT>
__global__ void __launch_bounds__(256) step_kernel_pipe(StepArgs a)
{
    __shared__ StepShared sh;
    step_prologue(a, sh);
    const XT *__restrict__ x = static_cast<const XT *>(a.x);
    const VT *__restrict__ vals = static_cast<const VT *>(a.A.vals);
    const uint16_t *__restrict__ codes = a.A.codes;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    AT ab_lane = 0, ex_lane = 0;
    for (int64_t q = warp0; q < a.A.n_slices; q += nwarps) {
        const int64_t b = q / kDirs;
        const int m = int(q - b * kDirs);
        const int64_t v = b * kSlice + lane;
        const int len4 = a.A.slice_len4[q];
        const int64_t base = a.A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup;
        const AT acc = row_dot_pipelined<VT, XT, AT>(vals, codes, base, len4, x, v, sh.delta);
        row_epilogue<XT, AT>(a, sh, q, lane, v, m, acc, ab_lane, ex_lane);
    }
    step_finish(a, sh, ab_lane, ex_lane);
}

// Variant 0: matrix streamed straight into registers (D groups prefetched).
template <class VT, class XT, class AT, int D>
__global__ void __launch_bounds__(256) step_kernel(StepArgs a)
{
    __shared__ StepShared sh;
    step_prologue(a, sh);
    const XT *__restrict__ x = static_cast<const XT *>(a.x);
    const VT *__restrict__ vals = static_cast<const VT *>(a.A.vals);
    const uint16_t *__restrict__ codes = a.A.codes;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    AT ab_lane = 0, ex_lane = 0;
    for (int64_t q = warp0; q < a.A.n_slices; q += nwarps) {
        const int64_t b = q / kDirs;
        const int m = int(q - b * kDirs);
        const int64_t v = b * kSlice + lane;
        const int len4 = a.A.slice_len4[q];
        const int64_t base = a.A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup;
        const AT acc = row_dot<VT, XT, AT, D>(vals, codes, base, len4, x, v, sh.delta);
        row_epilogue<XT, AT>(a, sh, q, lane, v, m, acc, ab_lane, ex_lane);
    }
    step_finish(a, sh, ab_lane, ex_lane);
}

// Variants 12-13: the registers path (one group in flight) with 32-bit
// slice, voxel and state indices.  A row streams from its own base
// pointers, so a group's address is one wide multiply-add, and a gather's
// index is one 32-bit add (states < 2^31, checked at launch).  Fewer
// instructions per nonzero and fewer live registers than variant 0; the
// block is held to 40 registers (six 256-thread CTAs per SM) or to 32
// (eight: every warp slot of the SM), trading spills for occupancy.
template <class VT, class XT, class AT>
__device__ __forceinline__ AT row_dot_lean(const VT *__restrict__ vrow, const uint16_t *__restrict__ crow, int len4,
                                           const XT *__restrict__ x, int vi, const int32_t *s_delta)
{
    constexpr int kStride = kSlice * kGroup;
    RawGroup<VT> nxt;
    Acc<AT> acc;
    if (len4 > 0) load_raw(vrow, crow, 0, nxt);
    for (int g = 0; g < len4; ++g) {
        const RawGroup<VT> cur = nxt;
        if (g + 1 < len4) load_raw(vrow, crow, (g + 1) * kStride, nxt);
        AT w[4];
        unpack(cur, w);
        const int c0 = int(cur.c.x & 0xffffu), c1 = int(cur.c.x >> 16);
        const int c2 = int(cur.c.y & 0xffffu), c3 = int(cur.c.y >> 16);
        const AT p0 = w[0] * AT(__ldg(x + (vi + s_delta[c0])));
        const AT p1 = w[1] * AT(__ldg(x + (vi + s_delta[c1])));
        const AT p2 = w[2] * AT(__ldg(x + (vi + s_delta[c2])));
        const AT p3 = w[3] * AT(__ldg(x + (vi + s_delta[c3])));
        acc.add((p0 + p1) + (p2 + p3));
    }
    return acc.value();
}

template <class VT, class XT, class AT, int MINB>
__global__ void __launch_bounds__(256, MINB) step_kernel_lean(StepArgs a)
{
    __shared__ StepShared sh;
    step_prologue(a, sh);
    const XT *__restrict__ x = static_cast<const XT *>(a.x);
    const VT *__restrict__ vals = static_cast<const VT *>(a.A.vals);
    const uint16_t *__restrict__ codes = a.A.codes;
    const int lane = threadIdx.x & 31;
    const int warp0 = int((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = int((gridDim.x * blockDim.x) >> 5);
    const int n_slices = int(a.A.n_slices);
    AT ab_lane = 0, ex_lane = 0;
    for (int q = warp0; q < n_slices; q += nwarps) {
        const int b = q / kDirs;
        const int m = q - b * kDirs;
        const int vi = b * kSlice + lane;
        const int len4 = a.A.slice_len4[q];
        const int64_t base = a.A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup;
        const AT acc = row_dot_lean<VT, XT, AT>(vals + base, codes + base, len4, x, vi, sh.delta);
        row_epilogue<XT, AT>(a, sh, q, lane, vi, m, acc, ab_lane, ex_lane);
    }
    step_finish(a, sh, ab_lane, ex_lane);
}

// Variants 10-11 and 14: K warps per slice (K = 2, 4, 8).  On small grids a slice
// per warp leaves most warp slots empty and each warp walks ~50 groups of
// its row one after another; splitting every slice's groups into K
// contiguous parts run by K warps of the CTA multiplies the matrix loads in
// flight by K.  The parts' sums meet in shared memory and warp part 0 adds
// them in part order (deterministic) and finishes the rows.
template <class VT, class XT, class AT, int K>
__global__ void __launch_bounds__(256) step_kernel_split(StepArgs a)
{
    __shared__ StepShared sh;
    __shared__ AT part[8][kSlice];
    step_prologue(a, sh);
    const XT *__restrict__ x = static_cast<const XT *>(a.x);
    const VT *__restrict__ vals = static_cast<const VT *>(a.A.vals);
    const uint16_t *__restrict__ codes = a.A.codes;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per_cta = (blockDim.x >> 5) / K;                 // slices per CTA round
    const int k = warp % K, slot = warp / K;
    const int64_t rounds = (a.A.n_slices + int64_t(gridDim.x) * per_cta - 1) / (int64_t(gridDim.x) * per_cta);
    AT ab_lane = 0, ex_lane = 0;
    for (int64_t rd = 0; rd < rounds; ++rd) {
        const int64_t q = (rd * gridDim.x + blockIdx.x) * per_cta + slot;
        const bool live = slot < per_cta && q < a.A.n_slices;
        AT acc = 0;
        int64_t b = 0, v = 0;
        int m = 0;
        if (live) {
            b = q / kDirs;
            m = int(q - b * kDirs);
            v = b * kSlice + lane;
            const int len4 = a.A.slice_len4[q];
            const int chunk = (len4 + K - 1) / K;
            const int g0 = k * chunk < len4 ? k * chunk : len4;
            const int g1 = g0 + chunk < len4 ? g0 + chunk : len4;
            const int64_t base = a.A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup + int64_t(g0) * (kSlice * kGroup);
            acc = row_dot<VT, XT, AT, 2>(vals, codes, base, g1 - g0, x, v, sh.delta);
        }
        part[warp][lane] = acc;
        __syncthreads();
        if (live && k == 0) {
            AT sum = part[warp][lane];
#pragma unroll
            for (int j = 1; j < K; ++j) sum += part[warp + j][lane];
            row_epilogue<XT, AT>(a, sh, q, lane, v, m, sum, ab_lane, ex_lane);
        }
        __syncthreads();
    }
    step_finish(a, sh, ab_lane, ex_lane);
}

// ---------------------------------------------------------------------------
// Shared-memory halo variant (grids with nx a multiple of 32): a CTA takes a
// whole 32-voxel block (one x-run at fixed y, z), stages the state of the
// block's 3x3 neighbouring x-runs, widened by one voxel at each end, for all
// 26 directions (26 x 9 x 34 values) in shared memory, and its W warps then
// compute the block's 26 slices with every x gather served from that halo.

constexpr int kHaloRow = 34;
constexpr int kHaloElems = kDirs * 9 * kHaloRow;

template <class VT, class XT, class AT, int W>
__global__ void __launch_bounds__(W * 32) step_kernel_halo(StepArgs a)
{
    __shared__ StepShared sh;
    __shared__ int32_t s_hoff[kCodes];
    __shared__ XT s_x[kHaloElems];
    step_prologue(a, sh);
    for (int c = threadIdx.x; c < kCodes; c += blockDim.x) {
        const int d = c / kDirs, n = c % kDirs;
        s_hoff[c] = ((n * 3 + d / 9) * 3 + d / 3 % 3) * kHaloRow + d % 3;
    }
    const XT *__restrict__ x = static_cast<const XT *>(a.x);
    const VT *__restrict__ vals = static_cast<const VT *>(a.A.vals);
    const uint16_t *__restrict__ codes = a.A.codes;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t n_blocks = a.A.n_slices / kDirs;
    const int bpl = a.nx / kSlice;                 // blocks per x-line
    AT ab_lane = 0, ex_lane = 0;
    for (int64_t b = blockIdx.x; b < n_blocks; b += gridDim.x) {
        const int xb = int(b % bpl) * kSlice;
        const int64_t yz = b / bpl;
        const int yy = int(yz % a.ny), zz = int(yz / a.ny);
        __syncthreads();                           // previous block done with s_x
        for (int i = threadIdx.x; i < kHaloElems; i += blockDim.x) {
            const int row = i / kHaloRow, col = i - row * kHaloRow;
            const int n = row / 9, dz = row / 3 % 3 - 1, dy = row % 3 - 1;
            const int gx = xb + col - 1, gy = yy + dy, gz = zz + dz;
            XT val = XT(0);
            if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz)
                val = x[int64_t(n) * a.V + (int64_t(gz) * a.ny + gy) * a.nx + gx];
            s_x[i] = val;
        }
        __syncthreads();
        for (int m = wib; m < kDirs; m += W) {
            const int64_t q = b * kDirs + m;
            const int64_t v = b * kSlice + lane;
            const int len4 = a.A.slice_len4[q];
            const int64_t base = a.A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup;
            Group<AT> nxt;
            if (len4 > 0) load_group(vals, codes, base, nxt);
            Acc<AT> acc;
            for (int g = 0; g < len4; ++g) {
                const Group<AT> cur = nxt;
                if (g + 1 < len4) load_group(vals, codes, base + int64_t(g + 1) * (kSlice * kGroup), nxt);
                const AT p0 = cur.w[0] * AT(s_x[s_hoff[cur.c[0]] + lane]);
                const AT p1 = cur.w[1] * AT(s_x[s_hoff[cur.c[1]] + lane]);
                const AT p2 = cur.w[2] * AT(s_x[s_hoff[cur.c[2]] + lane]);
                const AT p3 = cur.w[3] * AT(s_x[s_hoff[cur.c[3]] + lane]);
                acc.add((p0 + p1) + (p2 + p3));
            }
            row_epilogue<XT, AT>(a, sh, q, lane, v, m, acc.value(), ab_lane, ex_lane);
        }
    }
    step_finish(a, sh, ab_lane, ex_lane);
}

// ---------------------------------------------------------------------------
// Persistent multi-step kernel: one cooperative launch advances n_steps, with
// a grid-wide barrier between steps.  The barrier's wait is bounded: after
// spin_limit polls (or when another block has flagged an error) the block
// records the failure in a.err and every block leaves the step loop, so the
// host sees DRTS_ETIMEOUT and the context stays usable.

// bar[0] = arrivals of the current round, bar[1] = round counter
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, uint32_t limit, int *err,
                                             bool skip)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *round = bar + 1;
        const unsigned r0 = *round;
        __threadfence();                       // this block's writes before arriving
        if (skip) {
            ok = 0;                            // fault injection: never arrive
        } else if (atomicAdd(bar, 1u) + 1u == nblocks) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(const_cast<unsigned *>(round), 1u);
        } else {
            for (uint32_t i = 0; *round == r0; ++i) {
                if (i >= limit || *(volatile int *)err != 0) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (!ok && !skip) atomicExch(err, 1);
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// matrix groups the persistent kernel keeps in flight per lane (the launch
// path's best registers variant at full size prefetches two)
constexpr int kPersistDepth = 2;

// K > 1: as the split variants, K warps share each slice (grids too small to
// give every warp slot a slice), the parts meeting in shared memory in part
// order.
template <class VT, class XT, class AT, int K>
__global__ void __launch_bounds__(256) persistent_kernel(StepArgs a0, void *other, int64_t n_steps,
                                                         double *det_base, int64_t max_steps, unsigned *bar,
                                                         int fault_skip_barrier)
{
    __shared__ StepShared sh;
    __shared__ double pd_red[32];
    __shared__ AT part[K > 1 ? 8 : 1][kSlice];
    step_delta(a0, sh);
    const VT *__restrict__ vals = static_cast<const VT *>(a0.A.vals);
    const uint16_t *__restrict__ codes = a0.A.codes;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t k = 0; k < n_steps; ++k) {
        StepArgs a = a0;
        a.t = a0.t + k;
        a.x = (k & 1) ? other : a0.x;
        a.y = (k & 1) ? const_cast<void *>(a0.x) : other;
        a.det = (det_base && a.t < max_steps) ? det_base + a.t * a.n_patch : nullptr;
        step_sources(a, sh);
        const XT *x = static_cast<const XT *>(a.x);
        // point detectors of x(t): CTA b reads detectors b, b + grid, ...
        if (a.pd.n_det > 0 && a.pd.hist && a.t < max_steps)
            for (int d = blockIdx.x; d < a.pd.n_det; d += gridDim.x)
                point_detector_block<XT, true>(a, x, 0, d, pd_red);
        AT ab_lane = 0, ex_lane = 0;
        if constexpr (K == 1) {
            for (int64_t q = warp0; q < a.A.n_slices; q += nwarps) {
                const int64_t b = q / kDirs;
                const int m = int(q - b * kDirs);
                const int64_t v = b * kSlice + lane;
                const int len4 = a.A.slice_len4[q];
                const int64_t base = a.A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup;
                const AT acc = row_dot<VT, XT, AT, kPersistDepth, true>(vals, codes, base, len4, x, v, sh.delta);
                row_epilogue<XT, AT, true>(a, sh, q, lane, v, m, acc, ab_lane, ex_lane);
            }
        } else {
            const int per_cta = (blockDim.x >> 5) / K;
            const int kk = warp % K, slot = warp / K;
            const int64_t span = int64_t(gridDim.x) * per_cta;
            const int64_t rounds = (a.A.n_slices + span - 1) / span;
            for (int64_t rd = 0; rd < rounds; ++rd) {
                const int64_t q = (rd * gridDim.x + blockIdx.x) * per_cta + slot;
                const bool live = slot < per_cta && q < a.A.n_slices;
                AT acc = 0;
                int64_t v = 0;
                int m = 0;
                if (live) {
                    const int64_t b = q / kDirs;
                    m = int(q - b * kDirs);
                    v = b * kSlice + lane;
                    const int len4 = a.A.slice_len4[q];
                    const int chunk = (len4 + K - 1) / K;
                    const int g0 = kk * chunk < len4 ? kk * chunk : len4;
                    const int g1 = g0 + chunk < len4 ? g0 + chunk : len4;
                    const int64_t base =
                        a.A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup + int64_t(g0) * (kSlice * kGroup);
                    acc = row_dot<VT, XT, AT, kPersistDepth, true>(vals, codes, base, g1 - g0, x, v, sh.delta);
                }
                part[warp][lane] = acc;
                __syncthreads();
                if (live && kk == 0) {
                    AT sum = part[warp][lane];
#pragma unroll
                    for (int j = 1; j < K; ++j) sum += part[warp + j][lane];
                    row_epilogue<XT, AT, true>(a, sh, q, lane, v, m, sum, ab_lane, ex_lane);
                }
                __syncthreads();
            }
        }
        step_finish(a, sh, ab_lane, ex_lane);
        if (k + 1 < n_steps &&
            !grid_barrier(bar, gridDim.x, a.spin_limit, a.err, fault_skip_barrier && blockIdx.x == 0 && k == 0))
            break;
    }
}

// ---------------------------------------------------------------------------
// Variant 1: the matrix stream goes through shared memory by bulk async copy
// (cp.async.bulk, completion on an mbarrier).  Each warp owns S stages of G
// groups; lane 0 keeps S-1 chunks of its upcoming slices in flight while the
// warp consumes the current one, so the HBM latency is covered by copies in
// flight rather than by registers and resident warps.

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait for phase `parity` of bar.  Gives up after kSpinLimit polls
// (each poll may suspend the thread for a while inside try_wait).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <class VT, int G, int S>
struct TmaStages {
    static constexpr uint32_t kValBytes = G * kSlice * kGroup * sizeof(VT);
    static constexpr uint32_t kCodeBytes = G * kSlice * kGroup * sizeof(uint16_t);
    // per-warp region rounded to 128 B so every warp's stages stay 16-byte
    // aligned for the bulk copies
    static constexpr uint32_t kWarpBytes = (S * (kValBytes + kCodeBytes) + S * 8 + 127) / 128 * 128;
};

template <int G>
__device__ __forceinline__ int chunks_of(int len4) { return (len4 + G - 1) / G; }

template <class VT, class XT, class AT, int G, int S>
__global__ void __launch_bounds__(256) step_kernel_tma(StepArgs a)
{
    using St = TmaStages<VT, G, S>;
    __shared__ StepShared sh;
    extern __shared__ __align__(128) unsigned char dyn[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char *wbase = dyn + size_t(wib) * St::kWarpBytes;
    VT *sval = reinterpret_cast<VT *>(wbase);
    uint16_t *scode = reinterpret_cast<uint16_t *>(wbase + S * St::kValBytes);
    uint64_t *bar = reinterpret_cast<uint64_t *>(wbase + S * (St::kValBytes + St::kCodeBytes));
    if ((smem_u32(dyn) & 127u) != 0) {   // stage alignment the bulk copies need
        if (threadIdx.x == 0) atomicExch(a.err, 2);
        return;
    }
    if (lane == 0)
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    fence_proxy_async();
    step_prologue(a, sh);        // includes __syncthreads

    const XT *__restrict__ x = static_cast<const XT *>(a.x);
    const VT *__restrict__ vals = static_cast<const VT *>(a.A.vals);
    const uint16_t *__restrict__ codes = a.A.codes;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int64_t nsl = a.A.n_slices;

    // Issue cursor (lane 0 only): next chunk (iq, ic) to copy.  The slice
    // table entries of the slice after iq are loaded one slice early so the
    // copy issue never waits on a global load.
    int64_t iq = warp0, iptr = 0, nq = warp0, nptr = 0;
    int ic = 0, ilen4 = 0, nlen4 = 0;
    uint32_t issued = 0, consumed = 0;
    auto load_next = [&]() {
        if (nq < nsl) {
            nlen4 = a.A.slice_len4[nq];
            nptr = a.A.slice_ptr[nq];
        }
    };
    auto take_next = [&]() {     // move the cursor to slice nq
        iq = nq;
        ilen4 = nlen4;
        iptr = nptr;
        ic = 0;
        nq += nwarps;
        load_next();
    };
    auto issue = [&]() {
        // chunk (iq, ic) into stage issued % S
        const int g0 = ic * G;
        const int ng = ilen4 - g0 < G ? ilen4 - g0 : G;
        const int s = issued % S;
        const int64_t e0 = (iptr + g0) * (kSlice * kGroup);
        const uint32_t vb = uint32_t(ng) * kSlice * kGroup * sizeof(VT);
        const uint32_t cb = uint32_t(ng) * kSlice * kGroup * sizeof(uint16_t);
        // fault injection (tests): warp 0 never issues chunk number
        // fault_skip_chunk, so its wait on that stage must run out
        if (!(warp0 == 0 && int64_t(issued) == a.fault_skip_chunk)) {
            mbar_arrive_expect_tx(&bar[s], vb + cb);
            bulk_copy_g2s(sval + size_t(s) * G * kSlice * kGroup, vals + e0, vb, &bar[s]);
            bulk_copy_g2s(scode + size_t(s) * G * kSlice * kGroup, codes + e0, cb, &bar[s]);
        }
        ++issued;
        if (++ic * G >= ilen4)
            do take_next(); while (iq < nsl && ilen4 == 0);
    };
    if (lane == 0) {
        load_next();
        do take_next(); while (iq < nsl && ilen4 == 0);
        while (issued < uint32_t(S) && iq < nsl) issue();
    }
    __syncwarp();

    bool ok = true;
    AT ab_lane = 0, ex_lane = 0;
    int len4_next = warp0 < nsl ? a.A.slice_len4[warp0] : 0;
    for (int64_t q = warp0; q < nsl && ok; q += nwarps) {
        const int64_t b = q / kDirs;
        const int m = int(q - b * kDirs);
        const int64_t v = b * kSlice + lane;
        const int len4 = len4_next;
        if (q + nwarps < nsl) len4_next = a.A.slice_len4[q + nwarps];
        const int nch = chunks_of<G>(len4);
        Acc<AT> acc;
        for (int c = 0; c < nch; ++c) {
            const int s = consumed % S;
            ok = __all_sync(0xffffffffu, mbar_wait(&bar[s], (consumed / S) & 1u, a.spin_limit));
            if (!ok) break;
            const int ng = len4 - c * G < G ? len4 - c * G : G;
            const VT *sv = sval + size_t(s) * G * kSlice * kGroup + lane * kGroup;
            const uint16_t *sc = scode + size_t(s) * G * kSlice * kGroup + lane * kGroup;
#pragma unroll 4
            for (int g = 0; g < ng; ++g) {
                AT w[4];
                int cc[4];
                load4_smem(sv + g * (kSlice * kGroup), w);
                load_codes_smem(sc + g * (kSlice * kGroup), cc);
                const AT p0 = w[0] * AT(__ldg(x + (v + sh.delta[cc[0]])));
                const AT p1 = w[1] * AT(__ldg(x + (v + sh.delta[cc[1]])));
                const AT p2 = w[2] * AT(__ldg(x + (v + sh.delta[cc[2]])));
                const AT p3 = w[3] * AT(__ldg(x + (v + sh.delta[cc[3]])));
                acc.add((p0 + p1) + (p2 + p3));
            }
            __syncwarp();
            ++consumed;
            if (lane == 0 && iq < nsl) {
                fence_proxy_async();     // stage s was read by the generic proxy
                issue();
            }
            __syncwarp();
        }
        if (!ok) break;
        row_epilogue<XT, AT>(a, sh, q, lane, v, m, acc.value(), ab_lane, ex_lane);
    }
    if (!ok) {
        if (lane == 0) atomicExch(a.err, 1);
        // let every copy still in flight land before the block exits
        while (consumed < issued) {
            mbar_wait(&bar[consumed % S], (consumed / S) & 1u, a.spin_limit);
            ++consumed;
        }
    }
    step_finish(a, sh, ab_lane, ex_lane);
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

namespace {

// Launchable step variants: 0 = registers (LDG) path, 1/2 = bulk-copy paths
// with (G, S) = (8, 3) and (4, 4) stage shapes.
template <class VT, class XT, class AT, int G, int S>
struct TmaLaunch {
    static size_t dyn(int threads) { return size_t(TmaStages<VT, G, S>::kWarpBytes) * (threads / 32); }
    static cudaError_t prepare(int threads)
    {
        return cudaFuncSetAttribute(step_kernel_tma<VT, XT, AT, G, S>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn(threads)));
    }
    static int per_sm(int threads)
    {
        int n = 0;
        if (prepare(threads) != cudaSuccess) {
            cudaGetLastError();       // shape too large: clear the (non-sticky) error
            return 0;
        }
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel_tma<VT, XT, AT, G, S>, threads,
                                                          dyn(threads)) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return n;
    }
    static cudaError_t launch(const StepArgs &a, int blocks, int threads, cudaStream_t s)
    {
        cudaError_t e = prepare(threads);
        if (e != cudaSuccess) return e;
        step_kernel_tma<VT, XT, AT, G, S><<<blocks, threads, dyn(threads), s>>>(a);
        return cudaGetLastError();
    }
};

template <class VT, class XT, class AT, int D>
struct RegLaunch {
    static int per_sm(int threads)
    {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<VT, XT, AT, D>, threads, 0);
        return n;
    }
    static cudaError_t launch(const StepArgs &a, int blocks, int threads, cudaStream_t s)
    {
        step_kernel<VT, XT, AT, D><<<blocks, threads, 0, s>>>(a);
        return cudaGetLastError();
    }
};

// Halo variants run with W warps whatever thread count is asked for, and only
// on grids whose x-lines split into whole 32-voxel blocks.
template <class VT, class XT, class AT, int K>
struct SplitLaunch {
    static int per_sm(int threads)
    {
        if (threads < 32 * K) return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel_split<VT, XT, AT, K>, threads, 0) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return n;
    }
    static cudaError_t launch(const StepArgs &a, int blocks, int threads, cudaStream_t s)
    {
        step_kernel_split<VT, XT, AT, K><<<blocks, threads, 0, s>>>(a);
        return cudaGetLastError();
    }
};

template <class VT, class XT, class AT, int MINB>
struct LeanLaunch {
    static int per_sm(int threads)
    {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel_lean<VT, XT, AT, MINB>, threads, 0);
        return n;
    }
    static cudaError_t launch(const StepArgs &a, int blocks, int threads, cudaStream_t s)
    {
        // 32-bit indices: slices, voxels and states below 2^31
        if (a.A.n_slices >= (int64_t(1) << 31) || a.V * kDirs >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
        step_kernel_lean<VT, XT, AT, MINB><<<blocks, threads, 0, s>>>(a);
        return cudaGetLastError();
    }
};

template <class VT, class XT, class AT, int W>
struct HaloLaunch {
    static int per_sm(int threads)
    {
        (void)threads;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel_halo<VT, XT, AT, W>, W * 32, 0) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return n;
    }
    static cudaError_t launch(const StepArgs &a, int blocks, int threads, cudaStream_t s)
    {
        (void)threads;
        if (a.nx % kSlice != 0) return cudaErrorInvalidValue;
        step_kernel_halo<VT, XT, AT, W><<<blocks, W * 32, 0, s>>>(a);
        return cudaGetLastError();
    }
};

template <class VT, class XT, class AT>
struct PipeLaunch {
    static int per_sm(int threads)
    {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel_pipe<VT, XT, AT>, threads, 0);
        return n;
    }
    static cudaError_t launch(const StepArgs &a, int blocks, int threads, cudaStream_t s)
    {
        step_kernel_pipe<VT, XT, AT><<<blocks, threads, 0, s>>>(a);
        return cudaGetLastError();
    }
};

// Variant table: 0-2 registers path with prefetch depth 1, 2, 3;
// 3-6 bulk-copy path with stage shapes (G groups, S stages) = (8,3), (4,3),
// (4,4), (2,6); 7-8 state halo in shared memory; 9 both streams pipelined;
// 10-11 two or four warps per slice; 12-13 registers path with 32-bit
// indices at six or eight CTAs per SM; 14 eight warps per slice.
template <class VT, class XT, class AT>
struct Variants {
    static int per_sm(int variant, int threads)
    {
        switch (variant) {
        case 0: return RegLaunch<VT, XT, AT, 1>::per_sm(threads);
        case 1: return RegLaunch<VT, XT, AT, 2>::per_sm(threads);
        case 2: return RegLaunch<VT, XT, AT, 3>::per_sm(threads);
        case 3: return TmaLaunch<VT, XT, AT, 8, 3>::per_sm(threads);
        case 4: return TmaLaunch<VT, XT, AT, 4, 3>::per_sm(threads);
        case 5: return TmaLaunch<VT, XT, AT, 4, 4>::per_sm(threads);
        case 6: return TmaLaunch<VT, XT, AT, 2, 6>::per_sm(threads);
        case 7: return HaloLaunch<VT, XT, AT, 13>::per_sm(threads);
        case 8: return HaloLaunch<VT, XT, AT, 26>::per_sm(threads);
        case 9: return PipeLaunch<VT, XT, AT>::per_sm(threads);
        case 10: return SplitLaunch<VT, XT, AT, 2>::per_sm(threads);
        case 11: return SplitLaunch<VT, XT, AT, 4>::per_sm(threads);
        case 12: return LeanLaunch<VT, XT, AT, 6>::per_sm(threads);
        case 13: return LeanLaunch<VT, XT, AT, 8>::per_sm(threads);
        case 14: return SplitLaunch<VT, XT, AT, 8>::per_sm(threads);
        }
        return 0;
    }
    static cudaError_t launch(int variant, const StepArgs &a, int blocks, int threads, cudaStream_t s)
    {
        switch (variant) {
        case 0: return RegLaunch<VT, XT, AT, 1>::launch(a, blocks, threads, s);
        case 1: return RegLaunch<VT, XT, AT, 2>::launch(a, blocks, threads, s);
        case 2: return RegLaunch<VT, XT, AT, 3>::launch(a, blocks, threads, s);
        case 3: return TmaLaunch<VT, XT, AT, 8, 3>::launch(a, blocks, threads, s);
        case 4: return TmaLaunch<VT, XT, AT, 4, 3>::launch(a, blocks, threads, s);
        case 5: return TmaLaunch<VT, XT, AT, 4, 4>::launch(a, blocks, threads, s);
        case 6: return TmaLaunch<VT, XT, AT, 2, 6>::launch(a, blocks, threads, s);
        case 7: return HaloLaunch<VT, XT, AT, 13>::launch(a, blocks, threads, s);
        case 8: return HaloLaunch<VT, XT, AT, 26>::launch(a, blocks, threads, s);
        case 9: return PipeLaunch<VT, XT, AT>::launch(a, blocks, threads, s);
        case 10: return SplitLaunch<VT, XT, AT, 2>::launch(a, blocks, threads, s);
        case 11: return SplitLaunch<VT, XT, AT, 4>::launch(a, blocks, threads, s);
        case 12: return LeanLaunch<VT, XT, AT, 6>::launch(a, blocks, threads, s);
        case 13: return LeanLaunch<VT, XT, AT, 8>::launch(a, blocks, threads, s);
        case 14: return SplitLaunch<VT, XT, AT, 8>::launch(a, blocks, threads, s);
        }
        return cudaErrorInvalidValue;
    }
};

using VarF64 = Variants<double, double, double>;
using VarF32 = Variants<float, float, float>;
using VarF16 = Variants<__half, float, float>;

}  // namespace

int step_default_blocks(int precision, int R, int threads, int variant)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    (void)R;
    int per_sm = precision == DRTS_FP64 ? VarF64::per_sm(variant, threads)
               : precision == DRTS_FP32 ? VarF32::per_sm(variant, threads)
                                        : VarF16::per_sm(variant, threads);
    return per_sm < 1 ? 0 : sms * per_sm;
}

namespace {
template <class VT, class XT, class AT, int K>
int persistent_fit(int threads)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, persistent_kernel<VT, XT, AT, K>, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <class VT, class XT, class AT>
int persistent_fit_k(int threads, int split)
{
    return split == 8 ? persistent_fit<VT, XT, AT, 8>(threads)
         : split == 4 ? persistent_fit<VT, XT, AT, 4>(threads)
         : split == 2 ? persistent_fit<VT, XT, AT, 2>(threads)
                      : persistent_fit<VT, XT, AT, 1>(threads);
}

template <class VT, class XT, class AT, int K>
cudaError_t persistent_launch(const StepArgs &a, void *other, int64_t n_steps, double *det_base,
                              int64_t max_steps, unsigned *bar, int fault, int blocks, int threads,
                              cudaStream_t s)
{
    StepArgs a0 = a;
    void *args[] = {&a0, &other, &n_steps, &det_base, &max_steps, &bar, &fault};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void *>(persistent_kernel<VT, XT, AT, K>), dim3(blocks),
                                       dim3(threads), args, 0, s);
}

template <class VT, class XT, class AT>
cudaError_t persistent_launch_k(int split, const StepArgs &a, void *other, int64_t n_steps, double *det_base,
                                int64_t max_steps, unsigned *bar, int fault, int blocks, int threads, cudaStream_t s)
{
    if (split == 8)
        return persistent_launch<VT, XT, AT, 8>(a, other, n_steps, det_base, max_steps, bar, fault, blocks, threads, s);
    if (split == 4)
        return persistent_launch<VT, XT, AT, 4>(a, other, n_steps, det_base, max_steps, bar, fault, blocks, threads, s);
    if (split == 2)
        return persistent_launch<VT, XT, AT, 2>(a, other, n_steps, det_base, max_steps, bar, fault, blocks, threads, s);
    return persistent_launch<VT, XT, AT, 1>(a, other, n_steps, det_base, max_steps, bar, fault, blocks, threads, s);
}
}  // namespace

int persistent_blocks(int precision, int threads, int split)
{
    int dev = 0, sms = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return 0;
    const int per = precision == DRTS_FP64 ? persistent_fit_k<double, double, double>(threads, split)
                  : precision == DRTS_FP32 ? persistent_fit_k<float, float, float>(threads, split)
                                           : persistent_fit_k<__half, float, float>(threads, split);
    return per * sms;
}

cudaError_t launch_persistent(const StepArgs &a, void *other, int64_t n_steps, double *det_base, int64_t max_steps,
                              unsigned *bar, int fault_skip_barrier, int blocks, int threads, int split, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (a.A.precision == DRTS_FP64)
        return persistent_launch_k<double, double, double>(split, a, other, n_steps, det_base, max_steps, bar,
                                                           fault_skip_barrier, blocks, threads, s);
    if (a.A.precision == DRTS_FP32)
        return persistent_launch_k<float, float, float>(split, a, other, n_steps, det_base, max_steps, bar,
                                                        fault_skip_barrier, blocks, threads, s);
    return persistent_launch_k<__half, float, float>(split, a, other, n_steps, det_base, max_steps, bar,
                                                     fault_skip_barrier, blocks, threads, s);
}

cudaError_t launch_step(const StepArgs &a, int variant, int blocks, int threads, cudaStream_t s)
{
    if (blocks < 1) return cudaErrorInvalidConfiguration;
    if (a.A.precision == DRTS_FP64) return VarF64::launch(variant, a, blocks, threads, s);
    if (a.A.precision == DRTS_FP32) return VarF32::launch(variant, a, blocks, threads, s);
    return VarF16::launch(variant, a, blocks, threads, s);
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
