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
// Number formats (rounding the dominant product only on exact grids):
//   * The tensor cores truncate FP32 accumulation unless every product of an
//     MMA lies on one grid; then the sum is exact.  So the dominant product is
//     made exact: a0 = A rounded to 8 bits on a grid shared by a block row
//     (quantum 2^(E-7), E = exponent of the row's largest value in the block)
//     and x0 = X rounded to 8 bits on a grid shared by the 26 directions of one
//     voxel and right-hand side; the products of one K = 32 block are integers
//     times one quantum below 2^21, exact in FP32.
//   * a1 = bf16(A - a0), a2 = bf16(A - a0 - a1) (A to ~25 bits: the stored FP32
//     value exactly in all but the smallest entries of a row) and
//     x1 = bf16(X - x0); the products with a1, a2 and x1 are 2^-7 of the result
//     or smaller, so their truncation is below 2^-31 relative.
//   * The state lives as the pair (x0, x1); every step writes it from the FP32
//     result.  Each tile's products are drained from tensor memory into FP32
//     sums on the CUDA cores (27 partials per output, plain round-to-nearest).
//   A CPU emulation of these formats on the FP64 oracle's matrix stays within
//   1.1e-5 relative L1 over 1500 steps (24^3 inclusions), below the 1e-4 bound.
//
// Kernel (one CTA per SM, persistent over output lines (y, z)): the state
// tile of input voxel i (64 right-hand sides of x0 and of x1 = 128 rows,
// 32 directions, bf16, 8 KB) feeds the three outputs on the output line whose
// neighbour it is.  Input columns are swept along x: each of the <= 9 input
// lines gives one tile per column.  Per tile:
//   MMA1  D[0:192)  = [x0; x1] (128 x 32) x [a0 of 3 outputs | a1 of 3 outputs]
//   MMA2  D[96:192) += [x0; x1] x [a2 of 3 outputs]
// (two K = 16 steps each), D in tensor memory, fresh per tile, double-buffered.
// Warp roles: warps 0-3 drain D (tcgen05.ld, lane quarter = warp) into FP32
// sums of the three live outputs and write each finished output voxel's new
// (x0, x1) tile; warp 4 issues the MMAs; warp 5 copies state tiles with
// cp.async.bulk; warps 6-7 expand A's union-dense values into the B operand
// tiles in shared memory.  B tiles are dedicated per input line role, whose
// sparsity never changes, so only the values are rewritten.  Every wait is on
// an mbarrier with a bounded poll count; a wait that runs out sets the
// context's error word and the CTA winds down.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "drts_device.cuh"
#include "drts_kernel_common.cuh"

namespace drts {
namespace {

constexpr int kTcK = 32;                      // directions padded to the K extent
constexpr int kXTileBytes = 8192;             // 128 rows x 32 directions x bf16
constexpr int kXSlots = 4;
constexpr int kB01 = 4 * 24 * 128;            // K 32 x N 192 (a0 | a1 of three outputs)
constexpr int kB2 = 4 * 12 * 128;             // K 32 x N 96 (a2 of three outputs)
constexpr int kBSlot = kB01 + kB2;
constexpr int kLines = 9;
constexpr int kOffX = kLines * kBSlot;                    // 165,888
constexpr int kOffXch = kOffX + kXSlots * kXTileBytes;    // 198,656
constexpr int kOffBar = kOffXch + 64 * 32 * 4;            // 206,848
constexpr int kSmemBytes = kOffBar + 512;
constexpr int kThreads = 256;
constexpr int kTmemCols = 512;
constexpr int kDCols = 192;

// barrier indices (8 bytes each at kOffBar)
constexpr int kBarBFull = 0, kBarBEmpty = 9, kBarXFull = 18, kBarXEmpty = 22, kBarDFull = 26, kBarDEmpty = 28;
constexpr int kNumBars = 30;

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

// kind::f16 instruction descriptor: bf16 A and B (K-major), FP32 D, M x N
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
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

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                   "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                   "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
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

// Split y into x0 (8 bits on the grid 2^(E-7) of the largest |y| of the tile
// row, E its exponent) and x1 = bf16(y - x0); write the row pair (x0 in row
// r, x1 in row 64 + r) of a state tile.
__device__ __forceinline__ void write_state_row(__nv_bfloat16 *tile, int r, const float y[kDirs])
{
    float mx = 0.0f;
#pragma unroll
    for (int m = 0; m < kDirs; ++m) mx = fmaxf(mx, fabsf(y[m]));
    int e = 0;
    frexpf(mx, &e);                                     // mx = f 2^e, f in [0.5, 1); e = 0 for mx = 0
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        __align__(16) __nv_bfloat16 h0[8], h1[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int n = g * 8 + k;
            float x0 = 0.0f, x1 = 0.0f;
            if (n < kDirs) {
                x0 = ldexpf(rintf(ldexpf(y[n], 8 - e)), e - 8);   // k 2^(e-8), |k| <= 256: exact
                x1 = y[n] - x0;                                  // exact
            }
            h0[k] = __float2bfloat16_rn(x0);
            h1[k] = __float2bfloat16_rn(x1);
        }
        *reinterpret_cast<uint4 *>(tile + xtile_elem(r, g * 8)) = *reinterpret_cast<const uint4 *>(h0);
        *reinterpret_cast<uint4 *>(tile + xtile_elem(64 + r, g * 8)) = *reinterpret_cast<const uint4 *>(h1);
    }
}

struct EpiState {
    float acc[3][kTcK];
};

// Add the drained tile (D buffer b) into the sums of the three outputs of
// column c: output c - 1 + bb sits in slot (c - 1 + bb) mod 3 = (ROT + 2 + bb) % 3.
template <int ROT>
__device__ __forceinline__ void drain_tile(EpiState &s, uint32_t tmem_q, int b)
{
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
        float dF[32], dS[32];
        tmem_ld32(tmem_q + uint32_t(b * kDCols + bb * 32), dF);
        tmem_ld32(tmem_q + uint32_t(b * kDCols + 96 + bb * 32), dS);
        tmem_wait_ld();
        constexpr int base = (ROT + 2) % 3;
        const int slot = (base + bb) % 3;
#pragma unroll
        for (int m = 0; m < kTcK; ++m) {
            if (slot == 0) s.acc[0][m] += dF[m] + dS[m];
            else if (slot == 1) s.acc[1][m] += dF[m] + dS[m];
            else s.acc[2][m] += dF[m] + dS[m];
        }
    }
}

template <int SLOT>
__device__ __forceinline__ void zero_slot(EpiState &s)
{
#pragma unroll
    for (int m = 0; m < kTcK; ++m) s.acc[SLOT][m] = 0.0f;
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
        __nv_bfloat16 *tile = static_cast<__nv_bfloat16 *>(a.y) + vox * (kXTileBytes / 2);
        write_state_row(tile, rhs, y);
    }
    named_sync(1, 128);
    zero_slot<SLOT>(s);
}

// Valid input lines (dy, dz) of output line (y, z), in role order L = (dz+1)*3 + (dy+1).
__device__ __forceinline__ int line_roles(int y, int z, int ny, int nz, int *Ls)
{
    int n = 0;
    for (int L = 0; L < kLines; ++L) {
        const int dy = L % 3 - 1, dz = L / 3 - 1;
        if (y + dy >= 0 && y + dy < ny && z + dz >= 0 && z + dz < nz) Ls[n++] = L;
    }
    return n;
}

template <int ROT>
__device__ __forceinline__ bool epi_column(EpiState &s, const StepArgs &a, int nL, uint32_t tmem_q,
                                           uint32_t bars, int64_t &tau, volatile int *abort, volatile int *failed)
{
    for (int li = 0; li < nL; ++li) {
        const int b = int(tau & 1);
        // every thread waits; a give-up anywhere is shared so the four warps agree
        if (!bar_wait(bars + 8 * (kBarDFull + b), uint32_t((tau >> 1) & 1), a.spin_limit, abort)) {
            *failed = 1;
            *abort = 1;
            atomicExch(a.err, 1);
        }
        named_sync(1, 128);
        if (*failed) return false;
        tc_fence_after();
        drain_tile<ROT>(s, tmem_q, b);
        tc_fence_before();
        bar_arrive(bars + 8 * (kBarDEmpty + b));
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
    const TcPlan &P = a.tcp;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int64_t n_lines = int64_t(ny) * nz;
    // an earlier launch gave up a wait: the state is already invalid, do nothing
    if (*reinterpret_cast<volatile int *>(a.err) != 0) return;

    // B tiles start at zero; positions outside the union are never written
    for (int i = tid; i < kLines * kBSlot / 16; i += kThreads) reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int L = 0; L < kLines; ++L) {
            bar_init(bars + 8 * (kBarBFull + L), 64);
            bar_init(bars + 8 * (kBarBEmpty + L), 1);
        }
        for (int s = 0; s < kXSlots; ++s) {
            bar_init(bars + 8 * (kBarXFull + s), 1);
            bar_init(bars + 8 * (kBarXEmpty + s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(bars + 8 * (kBarDFull + b), 1);
            bar_init(bars + 8 * (kBarDEmpty + b), 128);
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
            for (int m = 0; m < kTcK; ++m) s.acc[k][m] = 0.0f;
        const uint32_t tmem_q = tmem + (uint32_t(32 * warp) << 16);
        int64_t tau = 0;
        bool ok = true;
        for (int64_t line = blockIdx.x; line < n_lines && ok; line += gridDim.x) {
            const int y = int(line % ny), z = int(line / ny);
            int Ls[kLines];
            const int nL = line_roles(y, z, ny, nz, Ls);
            const int64_t row0 = (int64_t(z) * ny + y) * nx;
            for (int c = 0; c < nx && ok; ++c) {
                switch (c % 3) {
                case 0:
                    ok = epi_column<0>(s, a, nL, tmem_q, bars, tau, abort, failed);
                    if (!ok) break;
                    if (c >= 1) finalize<2>(s, a, xch, warp, lane, row0 + c - 1);
                    else zero_slot<2>(s);
                    if (c == nx - 1) { finalize<0>(s, a, xch, warp, lane, row0 + c); zero_slot<1>(s); }
                    break;
                case 1:
                    ok = epi_column<1>(s, a, nL, tmem_q, bars, tau, abort, failed);
                    if (!ok) break;
                    finalize<0>(s, a, xch, warp, lane, row0 + c - 1);
                    if (c == nx - 1) { finalize<1>(s, a, xch, warp, lane, row0 + c); zero_slot<2>(s); }
                    break;
                default:
                    ok = epi_column<2>(s, a, nL, tmem_q, bars, tau, abort, failed);
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
            const uint32_t id1 = idesc_bf16(128, 192), id2 = idesc_bf16(128, 96);
            const uint32_t xs0 = smem_u32(sm + kOffX), bs0 = smem_u32(sm);
            int64_t tau = 0;
            int u[kLines] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            bool ok = true;
            for (int64_t line = blockIdx.x; line < n_lines && ok; line += gridDim.x) {
                const int y = int(line % ny), z = int(line / ny);
                int Ls[kLines];
                const int nL = line_roles(y, z, ny, nz, Ls);
                for (int c = 0; c < nx && ok; ++c)
                    for (int li = 0; li < nL && ok; ++li) {
                        const int L = Ls[li];
                        const int sx = int(tau % kXSlots), b = int(tau & 1);
                        ok = bar_wait(bars + 8 * (kBarXFull + sx), uint32_t((tau / kXSlots) & 1), limit, abort) &&
                             bar_wait(bars + 8 * (kBarBFull + L), uint32_t(u[L] & 1), limit, abort) &&
                             (tau < 2 || bar_wait(bars + 8 * (kBarDEmpty + b), uint32_t(((tau >> 1) - 1) & 1), limit, abort));
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t d = tmem + uint32_t(b * kDCols);
                        const uint32_t xa = xs0 + sx * kXTileBytes, ba = bs0 + L * kBSlot;
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint64_t ad = smem_desc(xa + kk * 4096, 2048, 128);
                            mma_bf16(d, ad, smem_desc(ba + kk * 6144, 3072, 128), id1, kk);
                            mma_bf16(d + 96, ad, smem_desc(ba + kB01 + kk * 3072, 1536, 128), id2, 1);
                        }
                        mma_commit(bars + 8 * (kBarXEmpty + sx));
                        mma_commit(bars + 8 * (kBarBEmpty + L));
                        mma_commit(bars + 8 * (kBarDFull + b));
                        ++u[L];
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
                while (!bar_test(bars + 8 * (kBarDFull + int(last & 1)), uint32_t((last >> 1) & 1)) && spins < limit)
                    ++spins;
            }
        }
    } else if (warp == 5) {
        // ---- state tile copies (one thread) ----
        if (lane == 0) {
            const __nv_bfloat16 *x = static_cast<const __nv_bfloat16 *>(a.x);
            const uint32_t xs0 = smem_u32(sm + kOffX);
            int64_t tau = 0;
            bool ok = true;
            for (int64_t line = blockIdx.x; line < n_lines && ok; line += gridDim.x) {
                const int y = int(line % ny), z = int(line / ny);
                int Ls[kLines];
                const int nL = line_roles(y, z, ny, nz, Ls);
                for (int c = 0; c < nx && ok; ++c)
                    for (int li = 0; li < nL && ok; ++li) {
                        const int L = Ls[li];
                        const int sx = int(tau % kXSlots);
                        if (tau >= kXSlots &&
                            !bar_wait(bars + 8 * (kBarXEmpty + sx), uint32_t(((tau / kXSlots) - 1) & 1), limit, abort)) {
                            ok = false;
                            break;
                        }
                        const int64_t vi = (int64_t(z + L / 3 - 1) * ny + (y + L % 3 - 1)) * nx + c;
                        bar_expect_tx(bars + 8 * (kBarXFull + sx), kXTileBytes);
                        bulk_load(xs0 + sx * kXTileBytes, x + vi * (kXTileBytes / 2), kXTileBytes,
                                  bars + 8 * (kBarXFull + sx));
                        ++tau;
                    }
            }
            if (!ok) {
                *abort = 1;
                atomicExch(a.err, 1);
            }
        }
    } else {
        // ---- B operand tiles from A's union-dense values (64 threads) ----
        const int pt = tid - 192;
        int u[kLines] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        bool ok = true;
        for (int64_t line = blockIdx.x; line < n_lines && ok; line += gridDim.x) {
            const int y = int(line % ny), z = int(line / ny);
            int Ls[kLines];
            const int nL = line_roles(y, z, ny, nz, Ls);
            const int64_t row0 = (int64_t(z) * ny + y) * nx;
            for (int c = 0; c < nx && ok; ++c)
                for (int li = 0; li < nL && ok; ++li) {
                    const int L = Ls[li];
                    if (u[L] >= 1) {
                        if (!bar_wait(bars + 8 * (kBarBEmpty + L), uint32_t((u[L] - 1) & 1), limit, abort)) {
                            failed[1] = 1;
                            *abort = 1;
                            atomicExch(a.err, 1);
                        }
                        named_sync(2, 64);
                        if (failed[1]) {
                            ok = false;
                            break;
                        }
                    }
                    unsigned char *slot = sm + L * kBSlot;
#pragma unroll 1
                    for (int bb = 0; bb < 3; ++bb) {
                        const int j = c - 1 + bb;
                        // input voxel (c, line L) is neighbour (1 - bb, L) of output j
                        const int d = (L / 3) * 9 + (L % 3) * 3 + (2 - bb);
                        const int p0 = P.role_off[d], p1 = P.role_off[d + 1];
                        const bool valid = j >= 0 && j < nx;
                        const uint16_t *A0 = P.Au + (row0 + (valid ? j : 0)) * 3 * int64_t(P.U);
                        for (int p = p0 + pt; p < p1; p += 64) {
                            const uint32_t code = P.pos[p];
                            const int n = int(code >> 8), m = int(code & 255);
                            uint16_t v0 = 0, v1 = 0, v2 = 0;
                            if (valid) {
                                v0 = A0[p];
                                v1 = A0[P.U + p];
                                v2 = A0[2 * P.U + p];
                            }
                            const int q = bb * 4 + (m >> 3);
                            const int within = (m & 7) * 16 + (n & 7) * 2;
                            *reinterpret_cast<uint16_t *>(slot + ((n >> 3) * 24 + q) * 128 + within) = v0;
                            *reinterpret_cast<uint16_t *>(slot + ((n >> 3) * 24 + 12 + q) * 128 + within) = v1;
                            *reinterpret_cast<uint16_t *>(slot + kB01 + ((n >> 3) * 12 + q) * 128 + within) = v2;
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bar_arrive(bars + 8 * (kBarBFull + L));
                    ++u[L];
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

// Row (voxel j, direction m): per block role d the largest |value| fixes the
// grid of a0; every value is split into a0 + a1 + a2 and stored at its union
// position.
__global__ void tc_convert_kernel(SlicedMatrix A, int64_t V, const int16_t *pidx, int U, uint16_t *Au)
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
    uint16_t *out = Au + j * 3 * int64_t(U);
    for_row(A, q, lane, [&](int code, float v) {
        if (v == 0.0f) return;
        const int d = code / kDirs, n = code % kDirs;
        const int p = pidx[d * 676 + n * kDirs + m];
        if (p < 0) return;                      // cannot happen: the union covers every entry
        int e = 0;
        frexpf(rmax[d], &e);
        const float a0 = ldexpf(rintf(ldexpf(v, 8 - e)), e - 8);
        const float r1 = v - a0;
        const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(b1);
        out[p] = __bfloat16_as_ushort(__float2bfloat16_rn(a0));
        out[U + p] = __bfloat16_as_ushort(b1);
        out[2 * U + p] = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
    });
}

// ---- state layout helpers ----

__device__ __forceinline__ double tcx_value(const __nv_bfloat16 *x, int64_t v, int n, int r)
{
    const __nv_bfloat16 *t = x + v * (kXTileBytes / 2);
    return double(__bfloat162float(t[xtile_elem(r, n)])) + double(__bfloat162float(t[xtile_elem(64 + r, n)]));
}

__global__ void tcx_to_canonical_kernel(const __nv_bfloat16 *x, int64_t V, int r, double *out)
{
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= V * kDirs) return;
    out[s] = tcx_value(x, s / kDirs, int(s % kDirs), r);
}

__global__ void tcx_from_canonical_kernel(const double *in, int64_t V, int r, __nv_bfloat16 *x)
{
    const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= V) return;
    float y[kDirs];
    for (int n = 0; n < kDirs; ++n) y[n] = float(in[v * kDirs + n]);
    write_state_row(x + v * (kXTileBytes / 2), r, y);
}

__global__ void tcx_sum_kernel(const __nv_bfloat16 *x, int64_t V, int r, double *out)
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

// Ledger of X(t): one warp per voxel tile; lane k reads the 16-byte chunk k
// of each 512-byte group (rows rho .. of one direction group), so a warp
// reads the tile with coalesced loads; per right-hand side sums are
// collected in shared memory.
__global__ void __launch_bounds__(256) tcx_ledger_kernel(StepArgs a)
{
    __shared__ float red[2][64];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) (&red[0][0])[i] = 0.0f;
    __syncthreads();
    const __nv_bfloat16 *x = static_cast<const __nv_bfloat16 *>(a.x);
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    // chunk ch (0..511) of a tile is row ch % 8 of core matrix ch / 8 = (n group g, row
    // group h) -> rows rho = 8 h + ch % 8, directions 8 g .. 8 g + 7.  Lane l reads
    // chunks l + 32 k: its row's right-hand side rho & 63 depends only on k % 2.
    float ab[2] = {0.0f, 0.0f}, ex[2] = {0.0f, 0.0f};
    for (int64_t v = w0; v < a.V; v += nw) {
        const int k = a.med[v];
        const float abs_k = float(a.tab.absorb[k]);
        const int xx = int(v % a.nx), yy = int(v / a.nx % a.ny), zz = int(v / (int64_t(a.nx) * a.ny));
        const int mask = (zz == 0 ? 0 : (zz == a.nz - 1 ? 2 : 1)) * 9 + (yy == 0 ? 0 : (yy == a.ny - 1 ? 2 : 1)) * 3 +
                         (xx == 0 ? 0 : (xx == a.nx - 1 ? 2 : 1));
        const double *et = a.tab.exit_total + (k * 27 + mask) * kDirs;
        const uint4 *t = reinterpret_cast<const uint4 *>(x + v * (kXTileBytes / 2));
#pragma unroll 4
        for (int kc = 0; kc < 16; ++kc) {
            const int ch = lane + 32 * kc;
            const int n0 = (ch >> 7) * 8;
            const uint4 raw = t[ch];
            const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&raw);
            float s = 0.0f, se = 0.0f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int n = n0 + i;
                if (n >= kDirs) continue;
                const float xv = __bfloat162float(h[i]);
                s += xv;
                if (mask != 13) se += float(et[n]) * xv;
            }
            ab[kc & 1] += abs_k * s;
            ex[kc & 1] += se;
        }
    }
    for (int par = 0; par < 2; ++par) {
        const int ch = lane + 32 * par;
        const int rr = (((ch >> 3) & 15) * 8 + (ch & 7)) & 63;
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
    const __nv_bfloat16 *x = static_cast<const __nv_bfloat16 *>(a.x);
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

cudaError_t launch_tc_flags(const SlicedMatrix &A, int64_t V, uint8_t *flags, cudaStream_t s)
{
    const int64_t n = A.n_slices * kSlice;
    tc_flags_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(A, V, flags);
    return cudaGetLastError();
}

cudaError_t launch_tc_convert(const SlicedMatrix &A, int64_t V, const int16_t *pidx, int U, uint16_t *Au,
                              cudaStream_t s)
{
    const int64_t n = A.n_slices * kSlice;
    tc_convert_kernel<<<unsigned((n + 127) / 128), 128, 0, s>>>(A, V, pidx, U, Au);
    return cudaGetLastError();
}

int tc_blocks_per_sm()
{
    static bool attr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 0;
    }
    if (!attr[dev]) {
        if (cudaFuncSetAttribute(tcx_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        attr[dev] = true;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tcx_step_kernel, kThreads, kSmemBytes) != cudaSuccess) {
        cudaGetLastError();
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
    if (tc_blocks_per_sm() < 1) return cudaErrorInvalidConfiguration;
    const int64_t n_lines = int64_t(a.ny) * a.nz;
    const int grid = int(n_lines < sm_count() ? n_lines : sm_count());
    tcx_step_kernel<<<grid, kThreads, kSmemBytes, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tc_to_canonical(const void *x, int64_t V, int r, double *out, cudaStream_t s)
{
    const int th = 256;
    tcx_to_canonical_kernel<<<unsigned((V * kDirs + th - 1) / th), th, 0, s>>>(
        static_cast<const __nv_bfloat16 *>(x), V, r, out);
    return cudaGetLastError();
}

cudaError_t launch_tc_from_canonical(const double *in, int64_t V, int r, void *x, cudaStream_t s)
{
    const int th = 128;
    tcx_from_canonical_kernel<<<unsigned((V + th - 1) / th), th, 0, s>>>(in, V, r,
                                                                        static_cast<__nv_bfloat16 *>(x));
    return cudaGetLastError();
}

cudaError_t launch_tc_sum(const void *x, int64_t V, int r, double *out, cudaStream_t s)
{
    tcx_sum_kernel<<<sm_count() * 2, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(x), V, r, out);
    return cudaGetLastError();
}

}  // namespace drts
