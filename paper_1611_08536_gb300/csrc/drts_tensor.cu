// Tensor-core (tcgen05) form of the batched step X(t+1) = A X(t) + S(t).
//
// The 26 rows of output voxel j gather only from the 27 neighbouring voxels
// i = j + d, so
//     Y[j][m][r] = sum_d sum_n B_{j,d}[m][n] X[i][n][r],
// 27 small dense products (26 x 26 blocks times a 26 x R state tile).  Their
// sparsity pattern is the stencil's: over all voxels of a problem, block role d
// uses a fixed set U_d of (n, m) positions (5,504 in the interior plus the few
// that edge folding adds), so A is stored "union-dense": for every voxel and
// role the values at U_d, zeros where that voxel has none.
//
// Number formats (the dominant product is made exact):
//   * The tensor cores truncate FP32 accumulation unless every product of an
//     MMA lies on one grid; then the sum is exact.  A block row (voxel j, role
//     d, direction m) is scaled by 2^-Ea (Ea from the row's largest value) so
//     that a0 = rint(A 2^-Ea) is an integer of at most 256; a state row
//     (voxel i, right-hand side r) likewise by 2^-Ex, x0 = rint(X 2^-Ex).  The
//     products x0 a0 of one K = 32 block are integers below 2^21: exact.
//   * a1 = fp16(A 2^-Ea - a0), a2 = fp16(A 2^-Ea - a0 - a1) (A to ~30 bits) and
//     x1 = fp16(X 2^-Ex - x0) (11 bits of the residual); the products with
//     a1, a2 and x1 are 2^-8 of the result or smaller, so their truncation is
//     below 2^-32 relative.
//   * The state lives as (x0, x1, Ex); every step writes it from the FP32
//     result.  Each tile's products are drained from tensor memory, scaled by
//     2^(Ex + Ea) and added into FP32 sums on the CUDA cores (27 partials per
//     output, round to nearest).
//
// Kernel (one CTA per SM, persistent over output lines (y, z)): the state
// tile of input voxel i (64 right-hand sides of x0 and of x1 = 128 rows,
// 32 directions, fp16, 8 KB, Ex of row r stored at direction 26 of row r)
// feeds the three outputs on the output line whose neighbour it is.  Input
// columns are swept along x; each of the <= 9 input lines gives one tile per
// column.  The three outputs' 26 rows are packed into N = 80 columns
// (column 26 bb + m for output c - 1 + bb).  Per tile:
//   MMA1  D[0:160)  = [x0; x1] (128 x 32) x [a0 | a1]   (N = 160)
//   MMA2  D[80:160) += [x0; x1] x [a2]                 (N = 80)
// (two K = 16 steps each), D in tensor memory, fresh per tile, double-buffered.
// Warp roles: warps 0-3 drain D (tcgen05.ld, lane quarter = warp) into the
// FP32 sums of the three live outputs and write each finished output voxel's
// new tile; warp 4 issues the MMAs; warp 5 copies each tile's state and A
// chunks with cp.async.bulk into a ring of staging slots; warps 6-7 scatter
// the staged A values into the B operand tiles.  B tiles are dedicated per
// input line role, whose sparsity never changes, so only values are
// rewritten.  Every wait is on an mbarrier with a bounded poll count; a wait
// that runs out sets the context's error word and the CTA winds down.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <string>

#include "drts_device.cuh"
#include "drts_kernel_common.cuh"

namespace drts {
namespace {

constexpr int kTcK = 32;                      // directions padded to the K extent
constexpr int kN = 80;                        // three outputs x 26 rows, padded
constexpr int kXTileBytes = 8192;             // 128 rows x 32 directions x fp16
constexpr int kExpDir = 26;                   // direction slot holding Ex of a state row
// B operand tiles, K-major core matrices; consecutive direction groups are
// 16 bytes further apart than a whole group of core matrices, so the stores
// of one direction row to different groups fall in different banks
constexpr int kLbo01 = 20 * 128 + 16;         // K step of the (a0 | a1) tile, N 160
constexpr int kLbo2 = 10 * 128 + 16;          // K step of the a2 tile, N 80
constexpr int kB01 = 4 * kLbo01;              // K 32 x N 160 (a0 | a1)
constexpr int kB2 = 4 * kLbo2;                // K 32 x N 80 (a2)
constexpr int kBScale = kN * 4;               // 2^Ea per packed column
constexpr int kXScale = 64 * 4;               // 2^Ex of the tile's 64 state rows
constexpr int kBSlot = 16128;                 // kB01 + kB2 + kBScale + kXScale rounded to 128
constexpr int kLines = 9;
constexpr int kAStageMax = 8960;              // A chunks of one tile
constexpr int kRingSlot = kXTileBytes + kAStageMax;
constexpr int kRing = 4;
constexpr int kOffRing = kLines * kBSlot;                  // 145,152
constexpr int kOffXch = kOffRing + kRing * kRingSlot;      // 213,760
constexpr int kOffBar = kOffXch + kDirs * 64 * 4;          // 220,416
constexpr int kOffPos = kOffBar + 512;                     // the union position table
constexpr int kPosMax = 5760;                              // positions (padded) the table holds
constexpr int kSmemBytes = kOffPos + kPosMax * 2;
constexpr int kPrefetch = 8;                               // tiles whose data is pulled into L2 ahead
constexpr int kProducers = 128;               // threads expanding A into the B tiles (warps 6..9)
constexpr int kThreads = 192 + kProducers;
constexpr int kTmemCols = 512;
constexpr int kDCols = 160;
constexpr int kDBufs = 3;                     // accumulator buffers in tensor memory (480 of 512 columns)
constexpr int kExpBias = 160;                 // A row exponents are stored as Ea + 160 (uint8)

static_assert(kB01 + kB2 + kBScale + kXScale <= kBSlot, "B slot");
static_assert(kSmemBytes <= 232448, "shared memory");
// producer warp w expands the tiles staged in ring slot w: its waits on that
// slot's barriers then advance one phase at a time (an mbarrier parity wait
// must never run two phases ahead)
static_assert(kProducers / 32 == kRing, "one producer warp per staging slot");

// barrier indices (8 bytes each at kOffBar)
constexpr int kBarBFull = 0, kBarBEmpty = 9, kBarRFull = 18, kBarREmpty = 22, kBarDFull = 26, kBarDEmpty = 29;
constexpr int kNumBars = 32;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

// element offset of (row rho, direction n) in a state tile: K-major canonical
// layout of 8x8 core matrices, core matrix (n/8, rho/8) at (n/8 * 16 + rho/8) * 64
__host__ __device__ __forceinline__ int xtile_elem(int rho, int n)
{
    return (((n >> 3) * 16 + (rho >> 3)) * 64) + (rho & 7) * 8 + (n & 7);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return uint64_t((addr & 0x3FFFF) >> 4) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

// kind::f16 instruction descriptor: fp16 A and B (K-major), FP32 D, M x N
__device__ __forceinline__ uint32_t idesc_f16(int M, int N)
{
    return (1u << 4) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void bar_init(uint32_t bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint32_t bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 :: "r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait for the given phase parity of an mbarrier; gives up after
// `limit` polls or when another role has flagged an abort.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, uint32_t limit, volatile int *abort)
{
    for (uint32_t i = 0; i < limit; ++i) {
        if (bar_test(bar, parity)) return true;
        if (*abort) return false;
    }
    return false;
}

__device__ __forceinline__ void l2_prefetch(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(n) : "memory"); }

__device__ __forceinline__ double tc_source_value(const StepArgs &a, const SourceEntry &e)
{
    if (a.step_scale) return e.w * a.step_scale[e.rhs];
    const SourceProfile &p = a.prof[e.prof];
    if (a.t >= p.t0 && a.t < p.t0 + p.n_t) return e.w * a.prof_vals[p.off + (a.t - p.t0)];
    return 0.0;
}

// 2^k for -126 <= k <= 127 built from its bit pattern (exact), else 0 /
// infinity-free fallbacks through two factors
__device__ __forceinline__ float pow2f(int k)
{
    k = k < -126 ? -126 : (k > 127 ? 127 : k);
    return __int_as_float((k + 127) << 23);
}
// y * 2^k exactly for |k| <= 252 (two power-of-two factors, no intermediate overflow)
__device__ __forceinline__ float scale2(float y, int k)
{
    const int k1 = k / 2;
    return (y * pow2f(k1)) * pow2f(k - k1);
}

// Write row pair r / 64 + r of a state tile from y: Ex from the largest |y|
// (|y| 2^-Ex < 256), x0 = rint(y 2^-Ex) (exact in fp16), x1 = fp16(y 2^-Ex - x0),
// Ex itself (an integer, exact in fp16) at direction 26 of row r.
__device__ __forceinline__ void write_state_row(__half *tile, int r, const float y[kDirs])
{
    float mx = 0.0f;
#pragma unroll
    for (int m = 0; m < kDirs; ++m) mx = fmaxf(mx, fabsf(y[m]));
    int e = 0;
    frexpf(mx, &e);                                     // mx = f 2^e, f in [0.5, 1); e = 0 for mx = 0
    const int ex = e - 8;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        __align__(16) __half h0[8], h1[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int n = g * 8 + k;
            float x0 = 0.0f, x1 = 0.0f;
            if (n < kDirs) {
                const float ys = scale2(y[n], -ex);     // exact, |ys| < 256
                x0 = rintf(ys);
                x1 = ys - x0;                           // exact, |x1| <= 1/2
            } else if (n == kExpDir) {
                x0 = float(ex);
            }
            h0[k] = __float2half_rn(x0);
            h1[k] = __float2half_rn(x1);
        }
        *reinterpret_cast<uint4 *>(tile + xtile_elem(r, g * 8)) = *reinterpret_cast<const uint4 *>(h0);
        *reinterpret_cast<uint4 *>(tile + xtile_elem(64 + r, g * 8)) = *reinterpret_cast<const uint4 *>(h1);
    }
}

struct EpiState {
    float acc[3][kDirs];
};

// Add the drained tile (D buffer b) into the sums of the three outputs of
// column c: packed column q = 26 bb + m belongs to output c - 1 + bb, whose
// sums sit in slot (c - 1 + bb) mod 3 = (ROT + 2 + bb) % 3; scale 2^(Ex + Ea).
template <int ROT>
__device__ __forceinline__ void drain_tile(EpiState &s, uint32_t tmem_q, int b, float qx, const float *qa)
{
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        float dF[16], dS[16];
        tmem_ld16(tmem_q + uint32_t(b * kDCols + 16 * k), dF);
        tmem_ld16(tmem_q + uint32_t(b * kDCols + kN + 16 * k), dS);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int q = 16 * k + i;
            if (q >= 3 * kDirs) continue;
            const int bb = q / kDirs, m = q % kDirs;
            const int slot = (ROT + 2 + bb) % 3;
            const float v = (dF[i] + dS[i]) * (qx * qa[q]);
            if (slot == 0) s.acc[0][m] += v;
            else if (slot == 1) s.acc[1][m] += v;
            else s.acc[2][m] += v;
        }
    }
}

template <int SLOT>
__device__ __forceinline__ void zero_slot(EpiState &s)
{
#pragma unroll
    for (int m = 0; m < kDirs; ++m) s.acc[SLOT][m] = 0.0f;
}

// Output voxel j (sums in slot SLOT) is complete: combine the x0-row and
// x1-row sums of each right-hand side, add the sources, write the new tile.
template <int SLOT>
__device__ __forceinline__ void finalize(EpiState &s, const StepArgs &a, float *xch, int qd, int lane, int64_t vox)
{
    const int rhs = lane + 32 * (qd & 1);
    if (qd >= 2) {
#pragma unroll
        for (int m = 0; m < kDirs; ++m) xch[m * 64 + rhs] = s.acc[SLOT][m];
    }
    named_sync(1, 128);
    if (qd < 2) {
        float y[kDirs];
#pragma unroll
        for (int m = 0; m < kDirs; ++m) y[m] = s.acc[SLOT][m] + xch[m * 64 + rhs];
        if (a.n_src > 0 && a.src_voxel[vox]) {
            for (int e = 0; e < a.n_src; ++e) {
                const SourceEntry se = a.src[e];
                const int64_t sv = (int64_t(se.slice) / kDirs) * kSlice + se.lane;
                if (sv != vox || se.rhs != rhs) continue;
                const int sm = int(se.slice % kDirs);
                const float val = float(tc_source_value(a, se));
#pragma unroll
                for (int m = 0; m < kDirs; ++m)
                    if (m == sm) y[m] += val;
            }
        }
        __half *tile = static_cast<__half *>(a.y) + vox * (kXTileBytes / 2);
        write_state_row(tile, rhs, y);
    }
    named_sync(1, 128);
    zero_slot<SLOT>(s);
}

// Valid input lines (dy, dz) of output line (y, z) as a bit mask over the
// role order L = (dz+1)*3 + (dy+1).  (Masks, not arrays: small arrays indexed
// at run time live in local memory, which the large shared-memory carve-out
// leaves almost no L1 for.)
__device__ __forceinline__ uint32_t line_mask(int y, int z, int ny, int nz)
{
    uint32_t mask = 0;
#pragma unroll
    for (int L = 0; L < kLines; ++L) {
        const int dy = L % 3 - 1, dz = L / 3 - 1;
        if (y + dy >= 0 && y + dy < ny && z + dz >= 0 && z + dz < nz) mask |= 1u << L;
    }
    return mask;
}

template <int ROT>
__device__ __forceinline__ bool epi_column(EpiState &s, const StepArgs &a, uint32_t lmask, uint32_t tmem_q,
                                           unsigned char *sm, uint32_t bars, int64_t &tau, volatile int *abort,
                                           volatile int *failed, int rhs)
{
    const bool leader = (threadIdx.x & 31) == 0;
    for (int L = 0; L < kLines; ++L) {
        if (!((lmask >> L) & 1u)) continue;
        const int b = int(tau % kDBufs);
        // lane 0 of each warp waits; a give-up anywhere is shared so the four warps agree
        if (leader && !bar_wait(bars + 8 * (kBarDFull + b), uint32_t((tau / kDBufs) & 1), a.spin_limit, abort)) {
            *failed = 1;
            *abort = 1;
            atomicExch(a.err, 1);
        }
        named_sync(1, 128);
        if (*failed) return false;
        tc_fence_after();
        // the state rows' scales 2^Ex, copied into the B slot by its producer
        const float qx = reinterpret_cast<const float *>(sm + L * kBSlot + kB01 + kB2 + kBScale)[rhs];
        drain_tile<ROT>(s, tmem_q, b, qx, reinterpret_cast<const float *>(sm + L * kBSlot + kB01 + kB2));
        tc_fence_before();
        __syncwarp();
        if (leader) {
            bar_arrive(bars + 8 * (kBarDEmpty + b));
            bar_arrive(bars + 8 * (kBarBEmpty + L));   // the B slot's scales are read
        }
        ++tau;
    }
    return true;
}

__global__ void __launch_bounds__(kThreads, 1) tcx_step_kernel(StepArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bars = smem_u32(sm + kOffBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kOffBar + 8 * kNumBars);
    volatile int *abort = reinterpret_cast<volatile int *>(sm + kOffBar + 8 * kNumBars + 4);
    volatile int *failed = reinterpret_cast<volatile int *>(sm + kOffBar + 8 * kNumBars + 8);
    float *xch = reinterpret_cast<float *>(sm + kOffXch);
    uint16_t *spos = reinterpret_cast<uint16_t *>(sm + kOffPos);
    int *s_roff = reinterpret_cast<int *>(sm + kOffBar + 288);      // role position offsets [28]
    int *s_coff = s_roff + 28;                                       // role chunk byte offsets [28]
    const TcPlan &P = a.tcp;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int64_t n_lines = int64_t(ny) * nz;
    // an earlier launch gave up a wait: the state is already invalid, do nothing
    if (*reinterpret_cast<volatile int *>(a.err) != 0) return;

    // B tiles start at zero; positions outside the union are never written
    for (int i = tid; i < kLines * kBSlot / 16; i += kThreads) reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < P.role_off[kOffs]; i += kThreads) spos[i] = P.pos[i];
    for (int i = tid; i < 28; i += kThreads) {
        s_roff[i] = P.role_off[i];
        s_coff[i] = P.chunk_off[i];
    }
    if (tid == 0) {
        for (int L = 0; L < kLines; ++L) {
            bar_init(bars + 8 * (kBarBFull + L), 1);            // producers, after their own barrier
            bar_init(bars + 8 * (kBarBEmpty + L), 1 + 4);       // MMA done + each epilogue warp read the scales
        }
        for (int sl = 0; sl < kRing; ++sl) {
            bar_init(bars + 8 * (kBarRFull + sl), 1);
            bar_init(bars + 8 * (kBarREmpty + sl), 1 + 1);      // MMA read the state tile + A scattered
        }
        for (int b = 0; b < kDBufs; ++b) {
            bar_init(bars + 8 * (kBarDFull + b), 1);
            bar_init(bars + 8 * (kBarDEmpty + b), 4);           // each epilogue warp
        }
        *abort = 0;
        failed[0] = 0;
        failed[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t limit = a.spin_limit;

    if (warp < 4) {
        // ---- epilogue: drain tiles, finish output voxels ----
        EpiState s;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int m = 0; m < kDirs; ++m) s.acc[k][m] = 0.0f;
        const uint32_t tmem_q = tmem + (uint32_t(32 * warp) << 16);
        const int rhs = lane + 32 * (warp & 1);
        int64_t tau = 0;
        bool ok = true;
        for (int64_t line = blockIdx.x; line < n_lines && ok; line += gridDim.x) {
            const int y = int(line % ny), z = int(line / ny);
            const uint32_t lmask = line_mask(y, z, ny, nz);
            const int64_t row0 = (int64_t(z) * ny + y) * nx;
            for (int c = 0; c < nx && ok; ++c) {
                switch (c % 3) {
                case 0:
                    ok = epi_column<0>(s, a, lmask, tmem_q, sm, bars, tau, abort, failed, rhs);
                    if (!ok) break;
                    if (c >= 1) finalize<2>(s, a, xch, warp, lane, row0 + c - 1);
                    else zero_slot<2>(s);
                    if (c == nx - 1) { finalize<0>(s, a, xch, warp, lane, row0 + c); zero_slot<1>(s); }
                    break;
                case 1:
                    ok = epi_column<1>(s, a, lmask, tmem_q, sm, bars, tau, abort, failed, rhs);
                    if (!ok) break;
                    finalize<0>(s, a, xch, warp, lane, row0 + c - 1);
                    if (c == nx - 1) { finalize<1>(s, a, xch, warp, lane, row0 + c); zero_slot<2>(s); }
                    break;
                default:
                    ok = epi_column<2>(s, a, lmask, tmem_q, sm, bars, tau, abort, failed, rhs);
                    if (!ok) break;
                    finalize<1>(s, a, xch, warp, lane, row0 + c - 1);
                    if (c == nx - 1) { finalize<2>(s, a, xch, warp, lane, row0 + c); zero_slot<0>(s); }
                    break;
                }
            }
        }
    } else if (warp == 4) {
        // ---- MMA issue (one thread) ----
        if (lane == 0) {
            const uint32_t id1 = idesc_f16(128, 2 * kN), id2 = idesc_f16(128, kN);
            const uint32_t ring0 = smem_u32(sm + kOffRing), bs0 = smem_u32(sm);
            int64_t tau = 0;
            uint32_t upar = 0;                      // parity of each B slot's uses
            bool ok = true;
            for (int64_t line = blockIdx.x; line < n_lines && ok; line += gridDim.x) {
                const int y = int(line % ny), z = int(line / ny);
                const uint32_t lmask = line_mask(y, z, ny, nz);
                for (int c = 0; c < nx && ok; ++c)
                    for (int L = 0; L < kLines && ok; ++L) {
                        if (!((lmask >> L) & 1u)) continue;
                        const int sr = int(tau % kRing), b = int(tau % kDBufs);
                        ok = bar_wait(bars + 8 * (kBarRFull + sr), uint32_t((tau / kRing) & 1), limit, abort) &&
                             bar_wait(bars + 8 * (kBarBFull + L), (upar >> L) & 1u, limit, abort) &&
                             (tau < kDBufs ||
                              bar_wait(bars + 8 * (kBarDEmpty + b), uint32_t(((tau / kDBufs) - 1) & 1), limit, abort));
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t d = tmem + uint32_t(b * kDCols);
                        const uint32_t xa = ring0 + sr * kRingSlot, ba = bs0 + L * kBSlot;
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint64_t ad = smem_desc(xa + kk * 4096, 2048, 128);
                            mma_f16(d, ad, smem_desc(ba + kk * 2 * kLbo01, kLbo01, 128), id1, kk);
                            mma_f16(d + kN, ad, smem_desc(ba + kB01 + kk * 2 * kLbo2, kLbo2, 128), id2, 1);
                        }
                        mma_commit(bars + 8 * (kBarREmpty + sr));
                        mma_commit(bars + 8 * (kBarBEmpty + L));
                        mma_commit(bars + 8 * (kBarDFull + b));
                        upar ^= 1u << L;
                        ++tau;
                    }
            }
            if (!ok) {
                *abort = 1;
                atomicExch(a.err, 1);
            }
            // wait (bounded) for the last tile's products before leaving
            if (tau > 0) {
                const int64_t last = tau - 1;
                uint32_t spins = 0;
                while (!bar_test(bars + 8 * (kBarDFull + int(last % kDBufs)), uint32_t((last / kDBufs) & 1)) &&
                       spins < limit)
                    ++spins;
            }
        }
    } else if (warp == 5) {
        // ---- state tile and A chunk copies (one thread) ----
        if (lane == 0) {
            const __half *x = static_cast<const __half *>(a.x);
            const unsigned char *Au = reinterpret_cast<const unsigned char *>(P.Au);
            const uint32_t ring0 = smem_u32(sm + kOffRing);
            int64_t tau = 0;
            bool ok = true;
            for (int64_t line = blockIdx.x; line < n_lines && ok; line += gridDim.x) {
                const int y = int(line % ny), z = int(line / ny);
                const uint32_t lmask = line_mask(y, z, ny, nz);
                const int64_t row0 = (int64_t(z) * ny + y) * nx;
                for (int c = 0; c < 3 && c < nx; ++c) {
                    l2_prefetch(Au + (row0 + c) * P.voxel_bytes, uint32_t(P.voxel_bytes));
                    for (int L = 0; L < kLines && c < 2; ++L) {
                        if (!((lmask >> L) & 1u)) continue;
                        l2_prefetch(x + ((int64_t(z + L / 3 - 1) * ny + (y + L % 3 - 1)) * nx + c) * (kXTileBytes / 2),
                                    kXTileBytes);
                    }
                }
                for (int c = 0; c < nx && ok; ++c)
                    for (int L = 0; L < kLines && ok; ++L) {
                        if (!((lmask >> L) & 1u)) continue;
                        const int sr = int(tau % kRing);
                        if (tau >= kRing &&
                            !bar_wait(bars + 8 * (kBarREmpty + sr), uint32_t(((tau / kRing) - 1) & 1), limit, abort)) {
                            ok = false;
                            break;
                        }
                        const int64_t vi = (int64_t(z + L / 3 - 1) * ny + (y + L % 3 - 1)) * nx + c;
                        uint32_t bytes = kXTileBytes, stage = 0;
                        int chunk_len[3];
#pragma unroll
                        for (int bb = 0; bb < 3; ++bb) {
                            const int d = 3 * L + 2 - bb;
                            const int j = c - 1 + bb;
                            chunk_len[bb] = (j >= 0 && j < nx) ? s_coff[d + 1] - s_coff[d] : 0;
                            bytes += uint32_t(chunk_len[bb]);
                        }
                        // pull data two columns ahead into L2: the state tile of this line,
                        // and once per column the whole A of the voxel three columns on
                        if (c + 2 < nx) l2_prefetch(x + (vi + 2) * (kXTileBytes / 2), kXTileBytes);
                        if (L == __ffs(lmask) - 1 && c + 3 < nx)
                            l2_prefetch(Au + (row0 + c + 3) * P.voxel_bytes, uint32_t(P.voxel_bytes));
                        const uint32_t slot = ring0 + sr * kRingSlot;
                        const uint32_t fb = bars + 8 * (kBarRFull + sr);
                        bar_expect_tx(fb, bytes);
                        bulk_load(slot, x + vi * (kXTileBytes / 2), kXTileBytes, fb);
#pragma unroll
                        for (int bb = 0; bb < 3; ++bb) {
                            const int d = 3 * L + 2 - bb;
                            if (chunk_len[bb] > 0)
                                bulk_load(slot + kXTileBytes + stage,
                                          Au + (row0 + c - 1 + bb) * P.voxel_bytes + s_coff[d],
                                          uint32_t(chunk_len[bb]), fb);
                            stage += uint32_t(s_coff[d + 1] - s_coff[d]);
                        }
                        ++tau;
                    }
            }
            if (!ok) {
                *abort = 1;
                atomicExch(a.err, 1);
            }
        }
    } else {
        // ---- B operand tiles from the staged A chunks: producer warp w expands
        // the tiles of ring slot w (tau = w mod 4), one warp per tile, so four
        // tiles are expanded at once.  By the time its wait for the staged data
        // succeeds, the loader has been released by the tile four back, hence
        // the MMA and the epilogue have passed every earlier use of the tile's
        // B slot: the slot's barrier is at most one phase behind. ----
        const int pw = warp - 6, npw = kProducers / 32;
        uint32_t upar = 0, used = 0;            // parity of each B slot's uses, slots used
        int64_t tau = 0;
        bool ok = true;
        for (int64_t line = blockIdx.x; line < n_lines && ok; line += gridDim.x) {
            const int y = int(line % ny), z = int(line / ny);
            const uint32_t lmask = line_mask(y, z, ny, nz);
            for (int c = 0; c < nx && ok; ++c)
                for (int L = 0; L < kLines && ok; ++L) {
                    if (!((lmask >> L) & 1u)) continue;
                    const uint32_t par = (upar >> L) & 1u, was = (used >> L) & 1u;
                    upar ^= 1u << L;
                    used |= 1u << L;
                    const int64_t tme = tau++;
                    if (int(tme % npw) != pw) continue;
                    const int sr = int(tme % kRing);
                    if (lane == 0) {
                        bool w = bar_wait(bars + 8 * (kBarRFull + sr), uint32_t((tme / kRing) & 1), limit, abort);
                        if (w && was) w = bar_wait(bars + 8 * (kBarBEmpty + L), par ^ 1u, limit, abort);
                        if (!w) {
                            failed[1] = 1;
                            *abort = 1;
                            atomicExch(a.err, 1);
                        }
                    }
                    __syncwarp();
                    if (failed[1]) {
                        ok = false;
                        break;
                    }
                    unsigned char *slot = sm + L * kBSlot;
                    float *scale = reinterpret_cast<float *>(slot + kB01 + kB2);
                    {
                        // the state tile's row scales, for the epilogue (rows r and r + 32)
                        const __half *xt = reinterpret_cast<const __half *>(sm + kOffRing + sr * kRingSlot);
                        float *xs = reinterpret_cast<float *>(slot + kB01 + kB2 + kBScale);
                        xs[lane] = pow2f(int(__half2float(xt[xtile_elem(lane, kExpDir)])));
                        xs[lane + 32] = pow2f(int(__half2float(xt[xtile_elem(lane + 32, kExpDir)])));
                    }
                    const unsigned char *stage = sm + kOffRing + sr * kRingSlot + kXTileBytes;
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb) {
                        const int j = c - 1 + bb;
                        // input voxel (c, line L) is neighbour (1 - bb, L) of output j
                        const int d = 3 * L + 2 - bb;
                        const int p0 = s_roff[d], np = s_roff[d + 1] - p0;
                        const bool valid = j >= 0 && j < nx;
                        const __half *t0 = reinterpret_cast<const __half *>(stage);
                        const unsigned char *ea = stage + 6 * np;
                        // four positions per iteration: their loads are issued before any store
                        for (int p = lane; p < np; p += 4 * 32) {
                            uint32_t code[4];
                            __half v0[4], v1[4], v2[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const int pk = p + 32 * k;
                                code[k] = pk < np ? uint32_t(spos[p0 + pk]) : 0xFFFFu;
                                v0[k] = v1[k] = v2[k] = __float2half_rn(0.0f);
                                if (valid && pk < np) {
                                    v0[k] = t0[pk];
                                    v1[k] = t0[np + pk];
                                    v2[k] = t0[2 * np + pk];
                                }
                            }
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                if (code[k] == 0xFFFFu) continue;
                                const int n = int(code[k] >> 8), q = bb * kDirs + int(code[k] & 255);
                                const int within = (q >> 3) * 128 + (q & 7) * 16 + (n & 7) * 2;
                                *reinterpret_cast<__half *>(slot + (n >> 3) * kLbo01 + within) = v0[k];
                                *reinterpret_cast<__half *>(slot + (n >> 3) * kLbo01 + 10 * 128 + within) = v1[k];
                                *reinterpret_cast<__half *>(slot + kB01 + (n >> 3) * kLbo2 + within) = v2[k];
                            }
                        }
                        if (lane < kDirs) scale[bb * kDirs + lane] = valid ? pow2f(int(ea[lane]) - kExpBias) : 0.0f;
                        stage += s_coff[d + 1] - s_coff[d];
                    }
                    // this warp's stores are made visible to the tensor cores, then its
                    // lane 0 signals the tile
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) {
                        bar_arrive(bars + 8 * (kBarBFull + L));
                        bar_arrive(bars + 8 * (kBarREmpty + sr));
                    }
                }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols));
    }
}

// ---- assembly of the union-dense A (once per problem) ----

// entries of the sliced row (slice q, lane): calls f(code, value) for each
// stored nonzero
template <class F>
__device__ __forceinline__ void for_row(const SlicedMatrix &A, int64_t q, int lane, F f)
{
    const int len = A.row_len[q * kSlice + lane];
    const int64_t base = A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup;
    const float *vals = static_cast<const float *>(A.vals);
    for (int e = 0; e < len; ++e) {
        const int64_t idx = base + int64_t(e / kGroup) * (kSlice * kGroup) + (e % kGroup);
        f(int(A.codes[idx]), vals[idx]);
    }
}

__global__ void tc_flags_kernel(SlicedMatrix A, int64_t V, uint8_t *flags)
{
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t q = g / kSlice;
    const int lane = int(g % kSlice);
    if (q >= A.n_slices || (q / kDirs) * kSlice + lane >= V) return;
    const int m = int(q % kDirs);
    for_row(A, q, lane, [&](int code, float v) {
        if (v != 0.0f) flags[(code / kDirs) * 676 + (code % kDirs) * kDirs + m] = 1;
    });
}

// Row (voxel j, direction m): per block role d, Ea from the row's largest
// |value| in the block; every value v becomes a0 = rint(v 2^-Ea) (|a0| <= 256),
// a1 = fp16(v 2^-Ea - a0), a2 = fp16(v 2^-Ea - a0 - a1), stored at its union
// position in the role's chunk, and Ea + 160 in the chunk's exponent bytes.
__global__ void tc_convert_kernel(SlicedMatrix A, int64_t V, const int16_t *pidx, TcPlan P, unsigned char *Au)
{
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t q = g / kSlice;
    const int lane = int(g % kSlice);
    if (q >= A.n_slices) return;
    const int64_t j = (q / kDirs) * kSlice + lane;
    if (j >= V) return;
    const int m = int(q % kDirs);
    float rmax[kOffs];
    for (int d = 0; d < kOffs; ++d) rmax[d] = 0.0f;
    for_row(A, q, lane, [&](int code, float v) {
        const int d = code / kDirs;
        rmax[d] = fmaxf(rmax[d], fabsf(v));
    });
    unsigned char *vox = Au + j * P.voxel_bytes;
    for (int d = 0; d < kOffs; ++d) {
        int e = 0;
        frexpf(rmax[d], &e);
        const int np = P.role_off[d + 1] - P.role_off[d];
        vox[P.chunk_off[d] + 6 * np + m] = uint8_t(e - 8 + kExpBias);
    }
    for_row(A, q, lane, [&](int code, float v) {
        if (v == 0.0f) return;
        const int d = code / kDirs, n = code % kDirs;
        const int p = pidx[d * 676 + n * kDirs + m];
        if (p < 0) return;                      // cannot happen: the union covers every entry
        int e = 0;
        frexpf(rmax[d], &e);
        const float vs = ldexpf(v, 8 - e);      // exact, |vs| < 256
        const float a0 = rintf(vs);
        const float r1 = vs - a0;               // exact
        const __half h1 = __float2half_rn(r1);
        const float r2 = r1 - __half2float(h1); // exact
        const int np = P.role_off[d + 1] - P.role_off[d];
        __half *t = reinterpret_cast<__half *>(vox + P.chunk_off[d]);
        t[p] = __float2half_rn(a0);
        t[np + p] = h1;
        t[2 * np + p] = __float2half_rn(r2);
    });
}

// ---- state layout helpers ----

__device__ __forceinline__ double tcx_value(const __half *x, int64_t v, int n, int r)
{
    const __half *t = x + v * (kXTileBytes / 2);
    const double s = ldexp(1.0, int(__half2float(t[xtile_elem(r, kExpDir)])));
    return (double(__half2float(t[xtile_elem(r, n)])) + double(__half2float(t[xtile_elem(64 + r, n)]))) * s;
}

__global__ void tcx_to_canonical_kernel(const __half *x, int64_t V, int r, double *out)
{
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= V * kDirs) return;
    out[s] = tcx_value(x, s / kDirs, int(s % kDirs), r);
}

__global__ void tcx_from_canonical_kernel(const double *in, int64_t V, int r, __half *x)
{
    const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= V) return;
    float y[kDirs];
    for (int n = 0; n < kDirs; ++n) y[n] = float(in[v * kDirs + n]);
    write_state_row(x + v * (kXTileBytes / 2), r, y);
}

__global__ void tcx_sum_kernel(const __half *x, int64_t V, int r, double *out)
{
    double acc = 0.0;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < V * kDirs;
         s += int64_t(gridDim.x) * blockDim.x)
        acc += tcx_value(x, s / kDirs, int(s % kDirs), r);
    acc = warp_sum(acc);
    __shared__ double smr[32];
    if ((threadIdx.x & 31) == 0) smr[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? smr[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) atomicAdd(out, t);
    }
}

// Ledger of X(t): one warp per voxel tile, coalesced 16-byte chunks.  Chunk
// ch (0..511) is row ch % 8 of core matrix ch / 8 = (direction group g, row
// group h): rows rho = 8 h + ch % 8, directions 8 g .. 8 g + 7.  Lane l reads
// chunks l + 32 k, whose right-hand side is l for even k and l + 32 for odd
// k; its two row scales sit in chunks 12 and 13 (direction 26 of rows l, l + 32).
__global__ void __launch_bounds__(256) tcx_ledger_kernel(StepArgs a)
{
    __shared__ float red[2][64];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) (&red[0][0])[i] = 0.0f;
    __syncthreads();
    const __half *x = static_cast<const __half *>(a.x);
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    float ab[2] = {0.0f, 0.0f}, ex[2] = {0.0f, 0.0f};
    for (int64_t v = w0; v < a.V; v += nw) {
        const int k = a.med[v];
        const float abs_k = float(a.tab.absorb[k]);
        const int xx = int(v % a.nx), yy = int(v / a.nx % a.ny), zz = int(v / (int64_t(a.nx) * a.ny));
        const int mask = (zz == 0 ? 0 : (zz == a.nz - 1 ? 2 : 1)) * 9 + (yy == 0 ? 0 : (yy == a.ny - 1 ? 2 : 1)) * 3 +
                         (xx == 0 ? 0 : (xx == a.nx - 1 ? 2 : 1));
        const double *et = a.tab.exit_total + (k * 27 + mask) * kDirs;
        const uint4 *t = reinterpret_cast<const uint4 *>(x + v * (kXTileBytes / 2));
        float sc[2];
#pragma unroll
        for (int par = 0; par < 2; ++par) {
            const uint4 raw = t[lane + 32 * (12 + par)];
            sc[par] = scale2(1.0f, int(__half2float(reinterpret_cast<const __half *>(&raw)[kExpDir - 24])));
        }
        float s[2] = {0.0f, 0.0f}, se[2] = {0.0f, 0.0f};
#pragma unroll 4
        for (int kc = 0; kc < 16; ++kc) {
            const int ch = lane + 32 * kc;
            const int n0 = (ch >> 7) * 8;
            const uint4 raw = t[ch];
            const __half *h = reinterpret_cast<const __half *>(&raw);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int n = n0 + i;
                if (n >= kDirs) continue;
                const float xv = __half2float(h[i]);
                s[kc & 1] += xv;
                if (mask != 13) se[kc & 1] += float(et[n]) * xv;
            }
        }
#pragma unroll
        for (int par = 0; par < 2; ++par) {
            ab[par] += abs_k * s[par] * sc[par];
            ex[par] += se[par] * sc[par];
        }
    }
    for (int par = 0; par < 2; ++par) {
        const int rr = lane + 32 * par;
        if (rr < a.R) {
            if (ab[par] != 0.0f) atomicAdd(&red[0][rr], ab[par]);
            if (ex[par] != 0.0f) atomicAdd(&red[1][rr], ex[par]);
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < a.R; r += blockDim.x) {
        if (red[0][r] != 0.0f) atomicAdd(&a.ledger[4 * r + 2], double(red[0][r]));
        if (red[1][r] != 0.0f) atomicAdd(&a.ledger[4 * r + 3], double(red[1][r]));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int e = 0; e < a.n_src; ++e) {
            const double val = tc_source_value(a, a.src[e]);
            if (val != 0.0) atomicAdd(&a.ledger[4 * a.src[e].rhs + 1], val);
        }
}

// Detector readout of X(t) (one block per patch, one thread per rhs, fixed order).
__global__ void tcx_det_kernel(StepArgs a)
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
    const __half *x = static_cast<const __half *>(a.x);
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
            for (int d = 0; d < kDirs; ++d) {
                const double ed = a.tab.exit_det[(k * 27 + mask) * kDirs + d];
                if (ed > 0.0) sum += ed * tcx_value(x, v, d, r);
            }
        }
    a.det[r * a.det_stride_r + p] = sum;
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

size_t tcx_state_bytes(int64_t V) { return size_t(V) * kXTileBytes; }
int tc_stage_limit() { return kAStageMax; }
int tc_position_limit() { return kPosMax; }

cudaError_t launch_tc_flags(const SlicedMatrix &A, int64_t V, uint8_t *flags, cudaStream_t s)
{
    const int64_t n = A.n_slices * kSlice;
    tc_flags_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(A, V, flags);
    return cudaGetLastError();
}

cudaError_t launch_tc_convert(const SlicedMatrix &A, int64_t V, const int16_t *pidx, const TcPlan &P,
                              void *Au, cudaStream_t s)
{
    const int64_t n = A.n_slices * kSlice;
    tc_convert_kernel<<<unsigned((n + 127) / 128), 128, 0, s>>>(A, V, pidx, P, static_cast<unsigned char *>(Au));
    return cudaGetLastError();
}

int tc_blocks_per_sm(std::string *why)
{
    static bool attr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        if (why) *why = "no current device";
        return 0;
    }
    if (!attr[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(tcx_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   kSmemBytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (why) *why = std::string("shared memory opt-in of ") + std::to_string(kSmemBytes) + " bytes: " +
                            cudaGetErrorString(e);
            return 0;
        }
        attr[dev] = true;
    }
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tcx_step_kernel, kThreads, kSmemBytes);
    if (e != cudaSuccess || n < 1) {
        cudaGetLastError();
        if (why) {
            cudaFuncAttributes fa{};
            cudaFuncGetAttributes(&fa, tcx_step_kernel);
            cudaGetLastError();
            *why = std::string("occupancy ") + (e == cudaSuccess ? "0" : cudaGetErrorString(e)) + ": " +
                   std::to_string(kThreads) + " threads x " + std::to_string(fa.numRegs) + " registers, " +
                   std::to_string(kSmemBytes) + " + " + std::to_string(fa.sharedSizeBytes) +
                   " bytes shared, kernel max threads " + std::to_string(fa.maxThreadsPerBlock);
        }
        return 0;
    }
    return n;
}

cudaError_t launch_tc_step(const StepArgs &a, bool functionals, cudaStream_t s)
{
    cudaError_t e;
    if (functionals) {
        if (a.det && a.n_patch > 0) {
            tcx_det_kernel<<<a.n_patch, kMaxRhs, 0, s>>>(a);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        tcx_ledger_kernel<<<unsigned(sm_count() * 4), 256, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (tc_blocks_per_sm(nullptr) < 1) return cudaErrorInvalidConfiguration;
    const int64_t n_lines = int64_t(a.ny) * a.nz;
    const int grid = int(n_lines < sm_count() ? n_lines : sm_count());
    tcx_step_kernel<<<grid, kThreads, kSmemBytes, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tc_to_canonical(const void *x, int64_t V, int r, double *out, cudaStream_t s)
{
    const int th = 256;
    tcx_to_canonical_kernel<<<unsigned((V * kDirs + th - 1) / th), th, 0, s>>>(static_cast<const __half *>(x), V,
                                                                                r, out);
    return cudaGetLastError();
}

cudaError_t launch_tc_from_canonical(const double *in, int64_t V, int r, void *x, cudaStream_t s)
{
    const int th = 128;
    tcx_from_canonical_kernel<<<unsigned((V + th - 1) / th), th, 0, s>>>(in, V, r, static_cast<__half *>(x));
    return cudaGetLastError();
}

cudaError_t launch_tc_sum(const void *x, int64_t V, int r, double *out, cudaStream_t s)
{
    tcx_sum_kernel<<<sm_count() * 2, 256, 0, s>>>(static_cast<const __half *>(x), V, r, out);
    return cudaGetLastError();
}

}  // namespace drts
