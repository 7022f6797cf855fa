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
//     MMA output lies on one grid; then the sum is exact.  A block row (voxel
//     j, role d, direction m) has an exponent Ea from its largest value, so
//     that a0 = rint(A 2^-Ea) is an integer of at most 256; a state row
//     (voxel i, right-hand side r) likewise Ex, x0 = rint(X 2^-Ex).  Both are
//     stored in bf16 WITH their power-of-two scale (a0 2^Ea, x0 2^Ex: at most
//     9 significant bits and the FP32 exponent range, so exact), hence every
//     product of output (r, m) of one tile lies on the grid 2^(Ex + Ea) and
//     their sum (below 2^21 grid units) is exact.  No scaling is left for the
//     drain.
//   * a1 = bf16(A - a0 2^Ea), a2 = bf16(A - a0 2^Ea - a1) (A to ~25 bits),
//     x1 = bf16(X - x0 2^Ex), x2 = bf16(X - x0 2^Ex - x1) (X to ~25 bits, and
//     to 16 bits for values far below their row's largest); their products
//     are 2^-8 of the result or smaller and accumulate in a second tensor-
//     memory sum, so their truncation is below 2^-32 relative.  Products of
//     two residual terms below 2^-24 relative (x1 a2 and smaller) that no MMA
//     forms for free are left out.
//   * The state lives as (x0 2^Ex, x1, x2); every step writes it from the
//     FP32 result.  Each tile's two sums are drained from tensor memory and
//     added into FP32 sums on the CUDA cores (27 partials per output, round
//     to nearest).  Rows whose largest |value| is below 2^-100 are stored as
//     zero (the bf16 terms would otherwise fall below the normal range).
//
// Kernel (one CTA per SM, persistent over output lines (y, z)): the state
// tile of input voxel i (x0, x1 and x2 of 64 right-hand sides, 32 directions,
// bf16, 12 KB) feeds the three outputs on the output line whose neighbour it
// is.  Input columns are swept along x; each of the <= 9 input lines gives
// one tile per column.  The three outputs' 26 rows are packed into N = 80
// columns (column 26 bb + m for output c - 1 + bb), and the B operand of a
// line holds [a0 | a1 | a2] side by side (N = 240).  Per tile, with M = 128
// rows and D fresh per tile in tensor memory (three buffers):
//   MMA1  D[0:160)  = [x0; x1] x [a0 | a1]   (N = 160)
//   MMA2  D[80:160) += [x0; x1] x [a2]       (N = 80)
//   MMA3  D[80:160) += [x1; x2] x [a0]       (N = 80)
// (two K = 16 steps each).  Right-hand side r then has x0 a0 exact in D row
// r, columns 0-79, and every other term once in rows r and 64 + r, columns
// 80-159 (row 64 + r of columns 0-79, x1 a0 again, is not read).  Warp roles:
// warps 0-3 drain D (tcgen05.ld, lane quarter = warp) into the FP32 sums of
// the three live outputs and write each finished output voxel's new tile;
// warp 11 issues the MMAs; warp 7 copies each tile's state and A chunks with
// cp.async.bulk into a ring of staging slots; warps 6-8 scatter the staged A
// values into the B operand tiles through a table of shared-memory offsets
// (one warp per tile).  B tiles are dedicated per input line role, whose
// sparsity never changes, so only values are rewritten.  Every wait is on an
// mbarrier with a bounded poll count (each poll may suspend the thread until
// the phase completes or a short hardware time limit passes); a wait that
// runs out sets the context's error word and the CTA winds down.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

#include "drts_device.cuh"
#include "drts_kernel_common.cuh"

namespace drts {
namespace {

constexpr int kN = 80;                        // three outputs x 26 rows, padded
constexpr int kXTileBytes = 12288;            // 3 terms x 64 rows x 32 directions x bf16
constexpr int kXGroup = 3072;                 // one direction group (8 directions) of a state tile
// B operand tile of a tile: [a0 | a1 | a2] side by side, N = 240 (30 groups of
// 8 columns), K-major core matrices; consecutive direction groups are 16
// bytes further apart than a whole group of core matrices, so the stores of
// one direction row to different groups fall in different banks
constexpr int kLbo = 30 * 128 + 16;           // K step (8 directions) of the B tile
constexpr int kA1Off = 10 * 128;              // a1 columns start 80 columns on
constexpr int kA2Off = 20 * 128;              // a2 columns start 160 columns on
constexpr int kBBytes = 15488;                // 4 K groups x kLbo, rounded to 128
constexpr int kLines = 9;
// Tile slots: state tile + B tile, from the copy until the MMAs are done.
// Staging slots: the tile's A chunks, from the copy until they are scattered.
constexpr int kSlots = 6;
constexpr int kSlotBytes = kXTileBytes + kBBytes;           // 27,776
constexpr int kStages = 5;
constexpr int kStageBytes = 8960;                           // A chunks of one tile
constexpr int kOffStage = kSlots * kSlotBytes;              // 166,656
constexpr int kOffXch = kOffStage + kStages * kStageBytes;  // 193,536
constexpr int kOffBar = kOffXch + kDirs * 64 * 4;           // 200,192
constexpr int kOffPos = kOffBar + 512;                      // the union offset table
constexpr int kPosMax = 5760;                               // positions (padded) the table holds
constexpr int kSmemBytes = kOffPos + kPosMax * 2;
// Warp roles.  A warp runs on scheduler warp % 4: one drain warp on each, the
// two copy warps (alternate tiles) and the MMA warp on schedulers 2 and 3, the
// five producers on the others' spare slots.
constexpr int kWarpLoad0 = 7, kWarpLoad1 = 10, kWarpMma = 11;
constexpr int kThreads = 12 * 32;
// producer index of warps 4, 5, 6, 8, 9 (-1: no producer role)
__device__ __forceinline__ int producer_of(int warp)
{
    return warp >= 4 && warp <= 6 ? warp - 4 : (warp == 8 || warp == 9 ? warp - 5 : -1);
}
static_assert(kStages == 5, "five producer warps, one per staging slot");
constexpr int kTmemCols = 512;
constexpr int kDCols = 160;
constexpr int kDBufs = 3;                     // accumulator buffers in tensor memory (480 of 512 columns)
constexpr int kTinyExp = -100;                // rows below 2^-100 are stored as zero

static_assert(4 * kLbo <= kBBytes && kBBytes % 128 == 0 && kSlotBytes % 128 == 0, "tile slot");
static_assert(kStageBytes % 128 == 0, "staging slot");
static_assert(kSmemBytes <= 232448, "shared memory");
static_assert(kN % 8 == 0 && 3 * kN == 240, "B tile column groups");
// Producer warp w expands the tiles staged in staging slot w, so its waits on
// that slot's barrier advance one phase at a time (an mbarrier parity wait
// must never run two phases ahead).  A tile slot is filled by different
// producer warps in turn, but in order: the loader copies into a tile slot
// only after the slot's previous MMAs, which waited for its previous B tile.
static_assert(kStages <= kSlots, "a tile waits for its staging slot before its tile slot is reused");

// barrier indices (8 bytes each at kOffBar)
constexpr int kBarXFull = 0;                  // [kSlots] state tile copied (transaction count)
constexpr int kBarBFull = 6;                  // [kSlots] B tile scattered
constexpr int kBarSDone = 12;                 // [kSlots] the tile's MMAs are done (slot free, products ready)
constexpr int kBarAFull = 18;                 // [kStages] A chunks copied (transaction count)
constexpr int kBarAEmpty = 23;                // [kStages] A chunks scattered
constexpr int kBarDEmpty = 28;                // [kDBufs] products drained
constexpr int kNumBars = 31;
static_assert(kBarBFull == kSlots && kBarAFull == 3 * kSlots && kBarDEmpty == kBarAFull + 2 * kStages &&
              kBarDEmpty + kDBufs == kNumBars && 8 * kNumBars + 16 <= 288, "barrier layout");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

// element offset of (row rho, direction n) in a state tile, rho = 64 t + r for
// term t of right-hand side r: K-major canonical layout of 8x8 core matrices,
// core matrix (n/8, rho/8) at (n/8 * 24 + rho/8) * 64.  A direction group holds
// the x0, x1 and x2 blocks one after the other, so rows [x0; x1] and rows
// [x1; x2] are both 128-row operands with the same strides.
__host__ __device__ __forceinline__ int xtile_elem(int rho, int n)
{
    return (((n >> 3) * 24 + (rho >> 3)) * 64) + (rho & 7) * 8 + (n & 7);
}

// byte offset of (direction n, packed column q) in a line's B tile
__device__ __forceinline__ int btile_byte(int n, int q)
{
    return (n >> 3) * kLbo + (q >> 3) * 128 + (q & 7) * 16 + (n & 7) * 2;
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

// The whole warp calls these with the same operands (they stay in uniform
// registers); one elected lane issues the instruction.
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p, e;\n\tsetp.ne.b32 p, %4, 0;\n\telect.sync _|e, 0xffffffff;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
                 "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}"
                 :: "r"(bar) : "memory");
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

// Whether the phase of the given parity has completed, without waiting.
__device__ __forceinline__ bool bar_done(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// One poll of an mbarrier phase: the thread may be suspended until the phase
// completes or a short hardware time limit passes, so a waiting warp takes
// few issue slots from the warps that share its scheduler.
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
    if (bar_done(bar, parity)) return true;         // the common case costs one instruction
    for (uint32_t i = 0; i < limit; ++i) {
        if (*abort) return false;
        if (bar_test(bar, parity)) return true;
    }
    return false;
}

// The same wait for a whole warp: every lane polls, then a warp vote makes
// the outcome uniform and brings the lanes back in step.  (Lanes that poll on
// their own can leave a wait at different times; a warp split that way must
// not reach an .aligned tcgen05 instruction, which needs every lane in step.)
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, uint32_t limit, volatile int *abort)
{
    return __all_sync(0xffffffffu, bar_wait(bar, parity, limit, abort));
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

// Write the three rows r, 64 + r, 128 + r of a state tile from y: Ex from
// the largest |y| (|y| 2^-Ex < 256), x0 = rint(y 2^-Ex) stored as x0 2^Ex
// (bf16, exact), x1 = bf16(y - x0 2^Ex), x2 = bf16(y - x0 2^Ex - x1); a row
// whose largest |y| is below 2^kTinyExp is stored as zero.
__device__ __forceinline__ void write_state_row(__nv_bfloat16 *tile, int r, const float y[kDirs])
{
    float mx = 0.0f;
#pragma unroll
    for (int m = 0; m < kDirs; ++m) mx = fmaxf(mx, fabsf(y[m]));
    int e = 0;
    frexpf(mx, &e);                                     // mx = f 2^e, f in [0.5, 1); e = 0 for mx = 0
    const int ex = e - 8;
    const bool tiny = e <= kTinyExp;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        __align__(16) __nv_bfloat16 h0[8], h1[8], h2[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int n = g * 8 + k;
            float x0 = 0.0f, r1 = 0.0f;
            if (n < kDirs && !tiny) {
                x0 = scale2(rintf(scale2(y[n], -ex)), ex);   // both scalings exact, |rint| <= 256
                r1 = y[n] - x0;                               // exact
            }
            h0[k] = __float2bfloat16_rn(x0);                  // exact
            h1[k] = __float2bfloat16_rn(r1);
            h2[k] = __float2bfloat16_rn(r1 - __bfloat162float(h1[k]));   // the difference is exact
        }
        *reinterpret_cast<uint4 *>(tile + xtile_elem(r, g * 8)) = *reinterpret_cast<const uint4 *>(h0);
        *reinterpret_cast<uint4 *>(tile + xtile_elem(64 + r, g * 8)) = *reinterpret_cast<const uint4 *>(h1);
        *reinterpret_cast<uint4 *>(tile + xtile_elem(128 + r, g * 8)) = *reinterpret_cast<const uint4 *>(h2);
    }
}

struct EpiState {
    float acc[3][kDirs];
};

// Registers written by tcgen05.ld are defined only after tcgen05.wait::ld;
// passing them through an empty asm after the wait keeps the compiler from
// moving their uses above it.
__device__ __forceinline__ void reg_fence(float (&v)[16])
{
    asm volatile("" : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]),
                 "+f"(v[7]), "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]),
                 "+f"(v[14]), "+f"(v[15]));
}

// Add columns 16 k .. 16 k + 15 of the drained tile into the sums of the
// three outputs of column c: packed column q = 26 bb + m belongs to output
// c - 1 + bb, whose sums sit in slot (c - 1 + bb) mod 3 = (ROT + 2 + bb) % 3.
// Column q of D holds the exact x0 a0 sum (lanes 0-63; lanes 64-127 hold x1
// a0, which the residual sums count already, and pass zeros), column 80 + q
// the residual terms' sum.
template <int ROT, int K>
__device__ __forceinline__ void add_part(EpiState &s, const float (&dF)[16], const float (&dS)[16])
{
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int q = 16 * K + i;
        if (q >= 3 * kDirs) continue;
        const int bb = q / kDirs, m = q % kDirs;
        const int slot = (ROT + 2 + bb) % 3;
        const float v = dF[i] + dS[i];
        if (slot == 0) s.acc[0][m] += v;
        else if (slot == 1) s.acc[1][m] += v;
        else s.acc[2][m] += v;
    }
}

__device__ __forceinline__ void load_part(uint32_t tmem_b, int k, bool with_f, float (&dF)[16], float (&dS)[16])
{
    if (with_f) {
        tmem_ld16(tmem_b + uint32_t(16 * k), dF);
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) dF[i] = 0.0f;
    }
    tmem_ld16(tmem_b + uint32_t(kN + 16 * k), dS);
}

__device__ __forceinline__ void wait_part(float (&dF)[16], float (&dS)[16])
{
    tmem_wait_ld();
    reg_fence(dF);
    reg_fence(dS);
}

// The five 16-column parts of a tile, software-pipelined: the loads of part
// k + 1 are in flight while part k is added.
template <int ROT>
__device__ __forceinline__ void drain_tile(EpiState &s, uint32_t tmem_b, bool with_f)
{
    float f0[16], s0[16], f1[16], s1[16];
    load_part(tmem_b, 0, with_f, f0, s0);
    wait_part(f0, s0);
    load_part(tmem_b, 1, with_f, f1, s1);
    add_part<ROT, 0>(s, f0, s0);
    wait_part(f1, s1);
    load_part(tmem_b, 2, with_f, f0, s0);
    add_part<ROT, 1>(s, f1, s1);
    wait_part(f0, s0);
    load_part(tmem_b, 3, with_f, f1, s1);
    add_part<ROT, 2>(s, f0, s0);
    wait_part(f1, s1);
    load_part(tmem_b, 4, with_f, f0, s0);
    add_part<ROT, 3>(s, f1, s1);
    wait_part(f0, s0);
    add_part<ROT, 4>(s, f0, s0);
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
    // the source flag is read before the barrier, which hides its latency
    const bool has_src = qd < 2 && a.n_src > 0 && a.src_voxel[vox];
    if (qd >= 2) {
#pragma unroll
        for (int m = 0; m < kDirs; ++m) xch[m * 64 + rhs] = s.acc[SLOT][m];
    }
    named_sync(1, 128);
    if (qd < 2) {
        float y[kDirs];
#pragma unroll
        for (int m = 0; m < kDirs; ++m) y[m] = s.acc[SLOT][m] + xch[m * 64 + rhs];
        if (has_src) {
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

// Drain the tiles of input column c (one per valid input line, in line
// order): each warp waits for the tile's products on its own (a warp-wide
// poll, so its lanes agree), adds them into its sums and releases the buffer.
// A tile's products are ready when its tile slot's MMAs are done; that
// barrier cannot run a phase ahead of this wait, because the slot's next
// tile needs the buffer that the drain of the tile after this one frees.
struct EpiPos {
    int sl, b;                                  // tile slot and accumulator buffer of the next tile
    uint32_t sph;                               // phase parity of the slot's current round
};

template <int ROT>
__device__ __forceinline__ bool epi_column(EpiState &s, const StepArgs &a, uint32_t lmask, uint32_t tmem_q,
                                           uint32_t bars, EpiPos &e, volatile int *abort, bool with_f)
{
    for (int L = 0; L < kLines; ++L) {
        if (!((lmask >> L) & 1u)) continue;
        const int b = e.b;
        if (!warp_wait(bars + 8 * (kBarSDone + e.sl), e.sph, a.spin_limit, abort)) {
            *abort = 1;
            if ((threadIdx.x & 31) == 0) atomicExch(a.err, 1);
            return false;
        }
        __syncwarp();
        tc_fence_after();
        drain_tile<ROT>(s, tmem_q + uint32_t(b * kDCols), with_f);
        tc_fence_before();
        __syncwarp();
        if ((threadIdx.x & 31) == 0) bar_arrive(bars + 8 * (kBarDEmpty + b));
        if (++e.b == kDBufs) e.b = 0;
        if (++e.sl == kSlots) { e.sl = 0; e.sph ^= 1u; }
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
    float *xch = reinterpret_cast<float *>(sm + kOffXch);
    uint16_t *spos = reinterpret_cast<uint16_t *>(sm + kOffPos);
    int *s_roff = reinterpret_cast<int *>(sm + kOffBar + 288);      // role position offsets [28]
    int *s_coff = s_roff + 28;                                       // role chunk byte offsets [28]
    const TcPlan &P = a.tcp;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int64_t n_lines = int64_t(ny) * nz;
    // an earlier launch gave up a wait: the state is already invalid, do nothing
    if (*reinterpret_cast<volatile int *>(a.err) != 0) return;

    // position (n, m) of role d = 3 L + 2 - bb lands in column q = 26 bb + m of
    // line L's B tile: its byte offset there
    for (int d = 0; d < kOffs; ++d) {
        const int bb = 2 - d % 3;
        for (int i = P.role_off[d] + tid; i < P.role_off[d + 1]; i += kThreads) {
            const int code = P.pos[i];
            spos[i] = uint16_t(btile_byte(code >> 8, bb * kDirs + (code & 255)));
        }
    }
    for (int i = tid; i < 28; i += kThreads) {
        s_roff[i] = P.role_off[i];
        s_coff[i] = P.chunk_off[i];
    }
    if (tid == 0) {
        for (int sl = 0; sl < kSlots; ++sl) {
            bar_init(bars + 8 * (kBarXFull + sl), 1);           // the loader's expect_tx
            bar_init(bars + 8 * (kBarBFull + sl), 1);           // the producer warp
            bar_init(bars + 8 * (kBarSDone + sl), 1);          // the MMAs' commit
        }
        for (int st = 0; st < kStages; ++st) {
            bar_init(bars + 8 * (kBarAFull + st), 1);           // the loader's expect_tx
            bar_init(bars + 8 * (kBarAEmpty + st), 1);          // the producer warp
        }
        for (int b = 0; b < kDBufs; ++b) bar_init(bars + 8 * (kBarDEmpty + b), 4);   // each epilogue warp
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == kWarpMma) {
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
        // ---- epilogue: drain tiles, finish output voxels.  The four warps run
        // the same loop to the end even after a failed wait (each later wait
        // then fails at once), so their named barriers always pair up. ----
        EpiState s;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int m = 0; m < kDirs; ++m) s.acc[k][m] = 0.0f;
        const uint32_t tmem_q = tmem + (uint32_t(32 * warp) << 16);
        const bool with_f = warp < 2;
        EpiPos ep{0, 0, 0u};
        for (int64_t line = blockIdx.x; line < n_lines; line += gridDim.x) {
            const int y = int(line % ny), z = int(line / ny);
            const uint32_t lmask = line_mask(y, z, ny, nz);
            const int64_t row0 = (int64_t(z) * ny + y) * nx;
            for (int c = 0; c < nx; ++c) {
                switch (c % 3) {
                case 0:
                    epi_column<0>(s, a, lmask, tmem_q, bars, ep, abort, with_f);
                    if (c >= 1) finalize<2>(s, a, xch, warp, lane, row0 + c - 1);
                    else zero_slot<2>(s);
                    if (c == nx - 1) { finalize<0>(s, a, xch, warp, lane, row0 + c); zero_slot<1>(s); }
                    break;
                case 1:
                    epi_column<1>(s, a, lmask, tmem_q, bars, ep, abort, with_f);
                    finalize<0>(s, a, xch, warp, lane, row0 + c - 1);
                    if (c == nx - 1) { finalize<1>(s, a, xch, warp, lane, row0 + c); zero_slot<2>(s); }
                    break;
                default:
                    epi_column<2>(s, a, lmask, tmem_q, bars, ep, abort, with_f);
                    finalize<1>(s, a, xch, warp, lane, row0 + c - 1);
                    if (c == nx - 1) { finalize<2>(s, a, xch, warp, lane, row0 + c); zero_slot<0>(s); }
                    break;
                }
            }
        }
    } else if (warp == kWarpMma) {
        // ---- MMA issue: the whole warp runs the loop in step (its values stay
        // warp-uniform), lane 0 issues the MMAs and commits ----
        const uint32_t id1 = idesc_bf16(128, 2 * kN), id2 = idesc_bf16(128, kN);
        // operand descriptors of tile slot 0 for the two K halves; tile slot sl
        // adds sl * kSlotBytes / 16 to their start-address field
        const uint32_t x0a = smem_u32(sm), b0a = x0a + kXTileBytes;
        uint64_t da01[2], da12[2], db0[2], db2[2];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            // rows [x0; x1] and rows [x1; x2] of directions 16 kk .. 16 kk + 15
            da01[kk] = smem_desc(x0a + kk * 2 * kXGroup, kXGroup, 128);
            da12[kk] = smem_desc(x0a + kk * 2 * kXGroup + 1024, kXGroup, 128);
            db0[kk] = smem_desc(b0a + kk * 2 * kLbo, kLbo, 128);
            db2[kk] = smem_desc(b0a + kA2Off + kk * 2 * kLbo, kLbo, 128);
        }
        int64_t tau = 0;
        int sl = 0, b = 0;
        uint32_t sph = 0, dph = 0;                  // phase parity of the current slot / buffer round
        bool ok = true;
        for (int64_t line = blockIdx.x; line < n_lines && ok; line += gridDim.x) {
            const int y = int(line % ny), z = int(line / ny);
            const uint32_t lmask = line_mask(y, z, ny, nz);
            for (int c = 0; c < nx && ok; ++c)
                for (int L = 0; L < kLines && ok; ++L) {
                    if (!((lmask >> L) & 1u)) continue;
                    const uint32_t bx = bars + 8 * (kBarXFull + sl), bbf = bars + 8 * (kBarBFull + sl),
                                   bde = bars + 8 * (kBarDEmpty + b);
                    // the three conditions are tested at once; only a tile that is
                    // not ready yet takes the polling path
                    const bool r = bar_done(bx, sph) & bar_done(bbf, sph) & (tau < kDBufs || bar_done(bde, dph ^ 1u));
                    if (!r)
                        ok = bar_wait(bx, sph, limit, abort) && bar_wait(bbf, sph, limit, abort) &&
                             (tau < kDBufs || bar_wait(bde, dph ^ 1u, limit, abort));
                    ok = __all_sync(0xffffffffu, ok);           // uniform, lanes in step for elect.sync
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t d = tmem + uint32_t(b * kDCols);
                    const uint64_t so = uint64_t(sl * (kSlotBytes >> 4));
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        mma_bf16(d, da01[kk] + so, db0[kk] + so, id1, kk);          // [a0 | a1]
                        mma_bf16(d + kN, da01[kk] + so, db2[kk] + so, id2, 1);      // a2
                        mma_bf16(d + kN, da12[kk] + so, db0[kk] + so, id2, 1);      // a0 of x1, x2
                    }
                    mma_commit(bars + 8 * (kBarSDone + sl));        // slot free, products ready
                    ++tau;
                    if (++sl == kSlots) { sl = 0; sph ^= 1u; }
                    if (++b == kDBufs) { b = 0; dph ^= 1u; }
                }
        }
        if (lane == 0) {
            if (!ok) {
                *abort = 1;
                atomicExch(a.err, 1);
            }
            // wait (bounded) for the last tile's products before leaving
            if (tau > 0) {
                const int64_t last = tau - 1;
                uint32_t spins = 0;
                while (!bar_test(bars + 8 * (kBarSDone + int(last % kSlots)), uint32_t((last / kSlots) & 1)) &&
                       spins < limit)
                    ++spins;
            }
        }
    } else if (warp == kWarpLoad0 || warp == kWarpLoad1) {
        // ---- state tile and A chunk copies: two warps take alternate tiles.
        // Lane 0 copies the state tile, lane 1 + 3 L + bb chunk bb of line L
        // (its offsets held in registers), lanes 28-29 issue the L2 prefetches:
        // each is one warp instruction with per-lane operands. ----
        const int me = warp == kWarpLoad0 ? 0 : 1;
        const __nv_bfloat16 *x = static_cast<const __nv_bfloat16 *>(a.x);
        const unsigned char *Au = reinterpret_cast<const unsigned char *>(P.Au);
        const uint32_t s0 = smem_u32(sm), st0 = smem_u32(sm + kOffStage);
        const int64_t vb = P.voxel_bytes;
        // this lane's chunk: line role my_l, output offset my_bb, role d = 3 L + 2 - bb
        const int my_l = (lane - 1) / 3, my_bb = (lane - 1) % 3;
        int my_len = 0, my_soff = 0, my_goff = 0;
        if (lane >= 1 && lane <= 3 * kLines) {
            const int d = 3 * my_l + 2 - my_bb;
            my_soff = s_coff[3 * my_l + 3] - s_coff[d + 1];      // chunks sit in bb order
            my_goff = s_coff[d];
            my_len = s_coff[d + 1] - s_coff[d];
        }
        int64_t tau = 0;
        int sl = 0, st = 0;
        uint32_t sph = 0, stph = 0;                 // phase parity of the current slot / stage round
        bool ok = true;
        for (int64_t line = blockIdx.x; line < n_lines && ok; line += gridDim.x) {
            const int y = int(line % ny), z = int(line / ny);
            const uint32_t lmask = line_mask(y, z, ny, nz);
            const int first_l = __ffs(lmask) - 1;
            const int64_t row0 = (int64_t(z) * ny + y) * nx;
            if (me == 0) {
                // the line's first columns into L2: A of voxels 0-2, state tiles of columns 0-1
                if (lane < 3 && lane < nx) l2_prefetch(Au + (row0 + lane) * vb, uint32_t(vb));
                if (lane >= 3 && lane < 3 + 2 * kLines) {
                    const int L = (lane - 3) % kLines, c = (lane - 3) / kLines;
                    if (((lmask >> L) & 1u) && c < nx)
                        l2_prefetch(x + ((int64_t(z + L / 3 - 1) * ny + (y + L % 3 - 1)) * nx + c) *
                                            (kXTileBytes / 2),
                                    kXTileBytes);
                }
            }
            for (int c = 0; c < nx && ok; ++c)
                for (int L = 0; L < kLines && ok; ++L) {
                    if (!((lmask >> L) & 1u)) continue;
                    const int tsl = sl, tst = st;
                    const uint32_t tsph = sph, tstph = stph;
                    const bool mine = (int(tau) & 1) == me;
                    const bool reuse_s = tau >= kSlots, reuse_a = tau >= kStages;
                    ++tau;
                    if (++sl == kSlots) { sl = 0; sph ^= 1u; }
                    if (++st == kStages) { st = 0; stph ^= 1u; }
                    if (!mine) continue;
                    // the tile slot's last MMAs and the staging slot's last scatter are done
                    if (lane == 0)
                        ok = (!reuse_s || bar_wait(bars + 8 * (kBarSDone + tsl), tsph ^ 1u, limit, abort)) &&
                             (!reuse_a || bar_wait(bars + 8 * (kBarAEmpty + tst), tstph ^ 1u, limit, abort));
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) break;
                    const int64_t vi = (int64_t(z + L / 3 - 1) * ny + (y + L % 3 - 1)) * nx + c;
                    const uint32_t xb = bars + 8 * (kBarXFull + tsl), ab = bars + 8 * (kBarAFull + tst);
                    // chunk bb of output c - 1 + bb exists inside the line only
                    const bool valid = my_l == L && c - 1 + my_bb >= 0 && c - 1 + my_bb < nx;
                    const int len = valid ? my_len : 0;
                    int bytes = __shfl_sync(0xffffffffu, len, 1 + 3 * L) + __shfl_sync(0xffffffffu, len, 2 + 3 * L) +
                                __shfl_sync(0xffffffffu, len, 3 + 3 * L);
                    if (lane == 0) {
                        bar_expect_tx(xb, kXTileBytes);
                        bar_expect_tx(ab, uint32_t(bytes));
                    }
                    __syncwarp();
                    uint32_t dst = st0 + tst * kStageBytes + my_soff, cb = ab, cl = uint32_t(len);
                    const void *src = Au + (row0 + c - 1 + my_bb) * vb + my_goff;
                    if (lane == 0) {
                        dst = s0 + tsl * kSlotBytes;
                        src = x + vi * (kXTileBytes / 2);
                        cl = kXTileBytes;
                        cb = xb;
                    }
                    if (cl > 0) bulk_load(dst, src, cl, cb);
                    // data ahead into L2: this line's state tile two columns on and,
                    // once per column, the whole A of the voxel three columns on
                    const void *pf = x + (vi + 2) * (kXTileBytes / 2);
                    uint32_t pl = (lane == 28 && c + 2 < nx) ? kXTileBytes : 0;
                    if (lane == 29) {
                        pf = Au + (row0 + c + 3) * vb;
                        pl = (L == first_l && c + 3 < nx) ? uint32_t(vb) : 0;
                    }
                    if (pl > 0) l2_prefetch(pf, pl);
                }
        }
        if (lane == 0) {
            if (!ok) {
                *abort = 1;
                atomicExch(a.err, 1);
            }
            // after a failed wait anywhere, copies this warp issued may never be
            // consumed: give them time to land (they cannot stall) before the
            // block exits
            if (*abort) {
                uint64_t t0, t1;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
                do {
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
                } while (t1 - t0 < 1000000u);
            }
        }
    } else if (producer_of(warp) >= 0) {
        // ---- B operand tiles from the staged A chunks: producer warp w expands
        // the tiles of staging slot w (tau = w mod kStages), one warp per tile,
        // so kStages tiles are expanded at once.  The tile's slot is free: the loader
        // waited for its last MMAs before the copies this warp waits for. ----
        const int pw = producer_of(warp);
        int sl = 0, st = 0;
        uint32_t stph = 0;                          // phase parity of the current stage round
        bool ok = true;
        for (int64_t line = blockIdx.x; line < n_lines && ok; line += gridDim.x) {
            const int y = int(line % ny), z = int(line / ny);
            const uint32_t lmask = line_mask(y, z, ny, nz);
            for (int c = 0; c < nx && ok; ++c)
                for (int L = 0; L < kLines && ok; ++L) {
                    if (!((lmask >> L) & 1u)) continue;
                    const int tsl = sl, tst = st;
                    const uint32_t tph = stph;
                    if (++sl == kSlots) sl = 0;
                    if (++st == kStages) { st = 0; stph ^= 1u; }
                    if (tst != pw) continue;
                    if (!bar_wait(bars + 8 * (kBarAFull + pw), tph, limit, abort)) {
                        *abort = 1;
                        if (lane == 0) atomicExch(a.err, 1);
                        ok = false;
                        break;
                    }
                    unsigned char *btile = sm + tsl * kSlotBytes + kXTileBytes;
                    // positions outside this line's union are zero
                    for (int i = lane; i < kBBytes / 16; i += 32)
                        reinterpret_cast<uint4 *>(btile)[i] = make_uint4(0, 0, 0, 0);
                    __syncwarp();
                    const unsigned char *stage = sm + kOffStage + pw * kStageBytes;
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb) {
                        // input voxel (c, line L) is neighbour (1 - bb, L) of output c - 1 + bb
                        const int d = 3 * L + 2 - bb;
                        const int p0 = s_roff[d], np = s_roff[d + 1] - p0;
                        const uint16_t *t = reinterpret_cast<const uint16_t *>(stage);
                        stage += s_coff[d + 1] - s_coff[d];
                        // an output outside the line: its chunk was not copied and its
                        // columns stay zero
                        const int j = c - 1 + bb;
                        if (j < 0 || j >= nx) continue;
                        // four positions per lane and pass: all loads before the stores
                        for (int p = lane; p < np; p += 4 * 32) {
                            uint32_t off[4];
                            uint16_t v0[4], v1[4], v2[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const int pk = p + 32 * k;
                                const bool in = pk < np;
                                off[k] = in ? uint32_t(spos[p0 + pk]) : 0xFFFFFFFFu;
                                v0[k] = in ? t[pk] : uint16_t(0);
                                v1[k] = in ? t[np + pk] : uint16_t(0);
                                v2[k] = in ? t[2 * np + pk] : uint16_t(0);
                            }
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                if (off[k] == 0xFFFFFFFFu) continue;
                                unsigned char *e = btile + off[k];
                                *reinterpret_cast<uint16_t *>(e) = v0[k];
                                *reinterpret_cast<uint16_t *>(e + kA1Off) = v1[k];
                                *reinterpret_cast<uint16_t *>(e + kA2Off) = v2[k];
                            }
                        }
                    }
                    // this warp's stores are made visible to the tensor cores, then its
                    // lane 0 signals the tile and frees the staging slot
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) {
                        bar_arrive(bars + 8 * (kBarBFull + tsl));
                        bar_arrive(bars + 8 * (kBarAEmpty + pw));
                    }
                }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kWarpMma) {
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
// |value| in the block (a0 = rint(v 2^-Ea) then has |a0| <= 256); every value
// v becomes a0 2^Ea, a1 = bf16(v - a0 2^Ea) and a2 = bf16(v - a0 2^Ea - a1),
// stored as bf16 at its union position in the role's chunk (three arrays of
// np values).  A block row whose largest |value| is below 2^kTinyExp is
// stored as zero.
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
    for_row(A, q, lane, [&](int code, float v) {
        if (v == 0.0f) return;
        const int d = code / kDirs, n = code % kDirs;
        const int p = pidx[d * 676 + n * kDirs + m];
        if (p < 0) return;                      // cannot happen: the union covers every entry
        int e = 0;
        frexpf(rmax[d], &e);
        if (e <= kTinyExp) return;
        const float a0 = scale2(rintf(scale2(v, 8 - e)), e - 8);   // exact, |rint| <= 256
        const float r1 = v - a0;                // exact
        const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(h1);  // exact
        const int np = P.role_off[d + 1] - P.role_off[d];
        __nv_bfloat16 *t = reinterpret_cast<__nv_bfloat16 *>(vox + P.chunk_off[d]);
        t[p] = __float2bfloat16_rn(a0);         // exact
        t[np + p] = h1;
        t[2 * np + p] = __float2bfloat16_rn(r2);
    });
}

// ---- state layout helpers ----

__device__ __forceinline__ double tcx_value(const __nv_bfloat16 *x, int64_t v, int n, int r)
{
    const __nv_bfloat16 *t = x + v * (kXTileBytes / 2);
    return double(__bfloat162float(t[xtile_elem(r, n)])) + double(__bfloat162float(t[xtile_elem(64 + r, n)])) +
           double(__bfloat162float(t[xtile_elem(128 + r, n)]));
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

// Ledger of X(t): one warp per voxel tile, coalesced 16-byte chunks.  Chunk
// ch (0..767) of a tile holds directions 8 g .. 8 g + 7 of row rho, with
// ch = 192 g + rho (rho = 64 term + r).  Lane l reads chunks l + 32 k,
// k = 0..23: direction group g = k / 6, row l + 32 (k mod 6), i.e. the x0,
// x1 and x2 rows of right-hand side l for even k and l + 32 for odd k.  All
// 24 loads of a tile are issued before any is used (12 KB per warp in
// flight).  Interior voxels with one absorption coefficient need only each
// right-hand side's sum over directions; boundary voxels (exit weights per
// direction) and per-direction absorption take the weighted form, which
// reads the tile's chunks a second time from cache.
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__global__ void __launch_bounds__(256, 2) tcx_ledger_kernel(StepArgs a)
{
    __shared__ float red[2][64];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) (&red[0][0])[i] = 0.0f;
    __syncthreads();
    const __nv_bfloat16 *x = static_cast<const __nv_bfloat16 *>(a.x);
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int64_t nxy = int64_t(a.nx) * a.ny;
    float ab[2] = {0.0f, 0.0f}, ex[2] = {0.0f, 0.0f};
    for (int64_t v = w0; v < a.V; v += nw) {
        const uint4 *t = reinterpret_cast<const uint4 *>(x + v * (kXTileBytes / 2));
        uint4 raw[24];
#pragma unroll
        for (int kc = 0; kc < 24; ++kc) raw[kc] = __ldcs(t + lane + 32 * kc);
        const int k = a.cls[v];
        // two-step interfaces: absorption per direction (s then sums it, not x)
        const double *ad = a.tab.absorb_dir ? a.tab.absorb_dir + k * kDirs : nullptr;
        const int zz = int(v / nxy), rem = int(v - zz * nxy);
        const int yy = rem / a.nx, xx = rem - yy * a.nx;
        const int mask = (zz == 0 ? 0 : (zz == a.nz - 1 ? 2 : 1)) * 9 + (yy == 0 ? 0 : (yy == a.ny - 1 ? 2 : 1)) * 3 +
                         (xx == 0 ? 0 : (xx == a.nx - 1 ? 2 : 1));
        if (!ad && mask == 13) {
            float s[2] = {0.0f, 0.0f};
#pragma unroll
            for (int kc = 0; kc < 24; ++kc) {
                const uint4 w = raw[kc];
                float cs = bf16_lo(w.x) + bf16_hi(w.x);         // directions 8 g, 8 g + 1
                if (kc < 18)                                     // g < 3: all eight are directions
                    cs += (bf16_lo(w.y) + bf16_hi(w.y)) + ((bf16_lo(w.z) + bf16_hi(w.z)) + (bf16_lo(w.w) + bf16_hi(w.w)));
                s[kc & 1] += cs;
            }
            const float abs_k = float(a.tab.absorb[k]);
            ab[0] += abs_k * s[0];
            ab[1] += abs_k * s[1];
        } else {
            const double *et = a.tab.exit_total + (k * 27 + mask) * kDirs;
            const float abs_k = float(a.tab.absorb[k]);
            float s[2] = {0.0f, 0.0f}, se[2] = {0.0f, 0.0f};
            // per direction group: its eight weights once, then its six chunks
            // (the tile's chunks again, from cache: indexing the register copy
            // with a loop counter would move it to local memory)
#pragma unroll 1
            for (int g = 0; g < 4; ++g) {
                float wa[8], we[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int n = 8 * g + i;
                    wa[i] = n < kDirs ? (ad ? float(ad[n]) : 1.0f) : 0.0f;
                    we[i] = n < kDirs && mask != 13 ? float(et[n]) : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    const uint4 w = __ldg(t + lane + 32 * (6 * g + j));
                    const uint32_t wd[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        if (8 * g + i >= kDirs) continue;       // padding columns of the last group
                        const float xv = (i & 1) ? bf16_hi(wd[i >> 1]) : bf16_lo(wd[i >> 1]);
                        s[j & 1] += wa[i] * xv;
                        se[j & 1] += we[i] * xv;
                    }
                }
            }
#pragma unroll
            for (int par = 0; par < 2; ++par) {
                ab[par] += ad ? s[par] : abs_k * s[par];
                ex[par] += se[par];
            }
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
    const __nv_bfloat16 *x = static_cast<const __nv_bfloat16 *>(a.x);
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
int tc_stage_limit() { return kStageBytes; }
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
        tcx_ledger_kernel<<<unsigned(sm_count() * 2), 256, 0, s>>>(a);     // two resident per SM
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
    tcx_to_canonical_kernel<<<unsigned((V * kDirs + th - 1) / th), th, 0, s>>>(static_cast<const __nv_bfloat16 *>(x), V,
                                                                                r, out);
    return cudaGetLastError();
}

cudaError_t launch_tc_from_canonical(const double *in, int64_t V, int r, void *x, cudaStream_t s)
{
    const int th = 128;
    tcx_from_canonical_kernel<<<unsigned((V + th - 1) / th), th, 0, s>>>(in, V, r, static_cast<__nv_bfloat16 *>(x));
    return cudaGetLastError();
}

cudaError_t launch_tc_sum(const void *x, int64_t V, int r, double *out, cudaStream_t s)
{
    tcx_sum_kernel<<<sm_count() * 2, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(x), V, r, out);
    return cudaGetLastError();
}

}  // namespace drts
