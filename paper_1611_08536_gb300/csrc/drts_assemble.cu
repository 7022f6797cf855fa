// Device assembler of the DRTS system matrix A (Eq. 18-23 of arXiv:1611.08536
// with the Section 4.2 edge and interface treatment), written straight into
// the sliced storage the step kernels stream.
//
// Rows are gathered, not scattered: row (voxel j, direction m) collects, for
// every neighbour voxel i = j + d (d in {-1,0,1}^3) and source direction n,
// the mass that state (i, n) sends to (j, m) in one step.  Entries come out in
// ascending (d, n), i.e. ascending canonical column.
//
//  * Plain rows (voxel off the grid edge whose 27 neighbours share one
//    refractive index) are a lookup of per-medium row templates.
//  * Other rows invert the folding of a raw contribution: a raw target can
//    reach (j, m) directly (possibly weakened by an interface transmission),
//    by Fresnel reflection at an interface from the voxel across it, or by
//    mirroring from outside the grid.
//  * With planar two-step interfaces, a source state whose direction reaches
//    the plane to the next z layer within the step uses that medium pair's
//    two-step entries instead of its medium's stencil: one part folds as
//    above, the part that already crossed (or reflected) at the plane folds
//    at the grid edge only.  Rows up to two layers from an index change are
//    therefore never plain.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>

#include "drts_device.cuh"

namespace drts {
namespace {

__constant__ int8_t c_dir[kDirs][3];
__constant__ int8_t c_nnzc[kDirs];
__constant__ int8_t c_dir_index[27];

cudaError_t upload_dirs()
{
    // __constant__ memory is per device: upload once on every device used
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    const Directions &D = dirs();
    int8_t v[kDirs][3], nz[kDirs], idx[27];
    for (int d = 0; d < kDirs; ++d) {
        for (int c = 0; c < 3; ++c) v[d][c] = int8_t(D.v[d][c]);
        nz[d] = int8_t(D.nnzc[d]);
    }
    for (int i = 0; i < 27; ++i) idx[i] = int8_t(D.index_of[i]);
    e = cudaMemcpyToSymbol(c_dir, v, sizeof(v));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_nnzc, nz, sizeof(nz));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_dir_index, idx, sizeof(idx));
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

__device__ __forceinline__ int vox_of(const DevTables &T, int x, int y, int z)
{
    return (z * T.ny + y) * T.nx + x;
}

constexpr size_t kStencil = size_t(kDirs) * kOffs * kDirs;   // one [26][27][26] raw stencil

// entry (n, o, m) of the raw stencil S ([26][27][26])
__device__ __forceinline__ double Wat(const double *S, int n, int o, int m)
{
    return __ldg(&S[(n * kOffs + o) * kDirs + m]);
}

// Two-step slot of source (voxel i of medium k, direction n): the pair
// (k, medium of the z layer S_n points to) when the indices differ and S_n
// reaches the plane between the layers within the step, else -1.
__device__ __forceinline__ int crossing_slot(const DevTables &T, const int i[3], int k, int n)
{
    if (!T.interface || c_dir[n][2] == 0) return -1;
    const int zn = i[2] + c_dir[n][2];
    if (zn < 0 || zn >= T.nz) return -1;
    const int p = __ldg(&T.pair_slot[k * T.K + T.med[vox_of(T, i[0], i[1], zn)]]);
    return p >= 0 && T.cross[p * kDirs + n] ? p : -1;
}

// incidence class of direction m on the face normal to axis a
__device__ __forceinline__ int inc_class(int m, int a)
{
    return c_dir[m][a] != 0 ? c_nnzc[m] : 0;
}

__device__ __forceinline__ int flip_dir(int m, int axes_mask)
{
    int v0 = c_dir[m][0], v1 = c_dir[m][1], v2 = c_dir[m][2];
    if (axes_mask & 1) v0 = -v0;
    if (axes_mask & 2) v1 = -v1;
    if (axes_mask & 4) v2 = -v2;
    return c_dir_index[(v2 + 1) * 9 + (v1 + 1) * 3 + (v0 + 1)];
}

// Face normal of an interface crossing from voxel i by offset o: the first
// axis with a nonzero offset whose axis-neighbour of i has another index,
// else the first axis with a nonzero offset.
__device__ int normal_axis(const DevTables &T, const int i[3], const int o[3], double ni)
{
    for (int a = 0; a < 3; ++a) {
        if (o[a] == 0) continue;
        int nb[3] = {i[0], i[1], i[2]};
        nb[a] += o[a];
        if (__ldg(&T.nref[T.med[vox_of(T, nb[0], nb[1], nb[2])]]) != ni) return a;
    }
    for (int a = 0; a < 3; ++a)
        if (o[a] != 0) return a;
    return 0;
}

// Mass that state (i, n) of medium k sends to (j, m) in one step, for a row
// voxel j that needs edge or interface folding.  The raw entries are the
// medium's stencil, or for a two-step crossing state the pair's entries that
// fold at edges and interfaces (S) plus those that fold at the grid edge
// only (S0).
__device__ double folded_contribution(const DevTables &T, const int i[3], int k, double ni,
                                      int n, const int j[3], int kj, double nj, int m)
{
    const int N[3] = {T.nx, T.ny, T.nz};
    const double *S = T.W + size_t(k) * kStencil;
    const double *S0 = nullptr;
    const int slot = crossing_slot(T, i, k, n);
    if (slot >= 0) {
        S = T.W2f + size_t(slot) * kStencil;
        S0 = T.W2n + size_t(slot) * kStencil;
    }
    double sum = 0.0;
    // (1) raw target (j, m): direct, or transmitted through an interface
    {
        const int o[3] = {j[0] - i[0], j[1] - i[1], j[2] - i[2]};
        if (S0) sum += Wat(S0, n, offset_index(o[0], o[1], o[2]), m);
        const double w = Wat(S, n, offset_index(o[0], o[1], o[2]), m);
        if (w > 0.0) {
            double f = 1.0;
            if ((o[0] | o[1] | o[2]) != 0 && nj != ni) {
                const int a = normal_axis(T, i, o, ni);
                if (c_dir[m][a] * o[a] > 0)
                    f = 1.0 - __ldg(&T.r_int[(size_t(k) * T.K + kj) * 4 + inc_class(m, a)]);
            }
            sum += w * f;
        }
    }
    // (2) reflection at an interface: raw target one voxel across, on axis a
    for (int a = 0; a < 3; ++a) {
        if (j[a] != i[a]) continue;
        for (int s = -1; s <= 1; s += 2) {
            int t[3] = {j[0], j[1], j[2]};
            t[a] += s;
            if (t[a] < 0 || t[a] >= N[a]) continue;
            const int kt = T.med[vox_of(T, t[0], t[1], t[2])];
            const double nt = __ldg(&T.nref[kt]);
            if (nt == ni) continue;
            const int o[3] = {t[0] - i[0], t[1] - i[1], t[2] - i[2]};
            if (normal_axis(T, i, o, ni) != a) continue;
            const int mr = flip_dir(m, 1 << a);
            if (c_dir[mr][a] * s <= 0) continue;
            const double w = Wat(S, n, offset_index(o[0], o[1], o[2]), mr);
            if (w > 0.0) sum += w * __ldg(&T.r_int[(size_t(k) * T.K + kt) * 4 + inc_class(mr, a)]);
        }
    }
    // (3) mirrored back from outside the grid across the faces in G
    int can = 0;
    for (int a = 0; a < 3; ++a)
        if (j[a] == i[a] && (j[a] == 0 || j[a] == N[a] - 1)) can |= 1 << a;
    for (int G = 1; G < 8; ++G) {
        if ((G & can) != G) continue;
        int t[3];
        for (int a = 0; a < 3; ++a)
            t[a] = (G >> a & 1) ? (j[a] == 0 ? -1 : N[a]) : j[a];
        const int o[3] = {t[0] - i[0], t[1] - i[1], t[2] - i[2]};
        const int mr = flip_dir(m, G);
        const int oi = offset_index(o[0], o[1], o[2]);
        const double w = Wat(S, n, oi, mr) + (S0 ? Wat(S0, n, oi, mr) : 0.0);
        if (w <= 0.0) continue;
        double f = 1.0;
        for (int a = 0; a < 3; ++a)
            if (G >> a & 1) f *= __ldg(&T.r_edge[k * 4 + inc_class(mr, a)]);
        sum += w * f;
    }
    return sum;
}

// Enumerate the nonzeros of row (voxel (x,y,z), direction m) in ascending
// column order; emit(code, value) with code = offset_index(d)*26 + n.
template <class Emit>
__device__ __forceinline__ void enumerate_row(const DevTables &T, int x, int y, int z, int m,
                                              Emit &emit)
{
    const int v = vox_of(T, x, y, z);
    if (T.plain[v]) {
        for (int d = 0; d < kOffs; ++d) {
            const int dx = d % 3 - 1, dy = d / 3 % 3 - 1, dz = d / 9 - 1;
            const int k = T.med[vox_of(T, x + dx, y + dy, z + dz)];
            const int32_t *off = T.tmpl_off + (size_t(k) * kDirs + m) * (kOffs + 1);
            const int e1 = __ldg(&off[d + 1]);
            for (int e = __ldg(&off[d]); e < e1; ++e)
                emit(d * kDirs + __ldg(&T.tmpl_n[e]), __ldg(&T.tmpl_val[e]));
        }
        return;
    }
    const int N[3] = {T.nx, T.ny, T.nz};
    const int j[3] = {x, y, z};
    const int kj = T.med[v];
    const double nj = __ldg(&T.nref[kj]);
    for (int d = 0; d < kOffs; ++d) {
        const int i[3] = {x + d % 3 - 1, y + d / 3 % 3 - 1, z + d / 9 - 1};
        if (i[0] < 0 || i[0] >= N[0] || i[1] < 0 || i[1] >= N[1] || i[2] < 0 || i[2] >= N[2]) continue;
        const int k = T.med[vox_of(T, i[0], i[1], i[2])];
        const double ni = __ldg(&T.nref[k]);
        for (int n = 0; n < kDirs; ++n) {
            const double val = folded_contribution(T, i, k, ni, n, j, kj, nj, m);
            if (val > 0.0) emit(d * kDirs + n, val);
        }
    }
}

__global__ void classify_kernel(DevTables T, uint8_t *plain)
{
    const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= T.V) return;
    const int x = int(v % T.nx), y = int(v / T.nx % T.ny), z = int(v / (int64_t(T.nx) * T.ny));
    uint8_t ok = x > 0 && y > 0 && z > 0 && x < T.nx - 1 && y < T.ny - 1 && z < T.nz - 1;
    if (ok) {
        const double n0 = T.nref[T.med[v]];
        for (int d = 0; d < kOffs && ok; ++d) {
            const int u = vox_of(T, x + d % 3 - 1, y + d / 3 % 3 - 1, z + d / 9 - 1);
            if (T.nref[T.med[u]] != n0) ok = 0;
        }
        // two-step interfaces: a source one layer above or below crosses when
        // the layer beyond it (two from the row) has another index
        for (int dz = -2; dz <= 2 && ok && T.interface; dz += 4)
            if (z + dz >= 0 && z + dz < T.nz && T.nref[T.med[vox_of(T, x, y, z + dz)]] != n0) ok = 0;
    }
    plain[v] = ok;
}

// FP16 tier: a value whose scaled size v / scale reaches kHalfSplitAt (the
// scale puts each direction's largest stencil value in (2^13, 2^14], so these
// are the few largest entries of a row, mostly the unscattered streaming ones)
// is stored as two FP16 terms with the same code, hi = RN(v/scale) and lo =
// RN(v/scale - hi): 21 significant bits instead of 11.  The step sums the two
// like any other entries; the export adds them back into one.
constexpr double kHalfSplitAt = 512.0;

struct CountEmit {
    double split_scale = 0.0;   // FP16: the row's scale; 0 = no split entries
    int count = 0;
    int split = 0;
    __device__ void operator()(int, double v)
    {
        ++count;
        if (split_scale > 0.0 && v / split_scale >= kHalfSplitAt) ++split;
    }
};

// one thread per row; a warp is exactly one slice
__global__ void count_kernel(DevTables T, int64_t n_slices, int32_t *row_len,
                             int32_t *slice_len4, unsigned long long *n_split)
{
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t q = g / kSlice;
    const int lane = int(g % kSlice);
    if (q >= n_slices) return;
    const int64_t b = q / kDirs;
    const int m = int(q % kDirs);
    const int64_t v = b * kSlice + lane;
    CountEmit ce;
    if (T.dir_scale) ce.split_scale = double(T.dir_scale[m]);
    if (v < T.V) {
        const int x = int(v % T.nx), y = int(v / T.nx % T.ny), z = int(v / (int64_t(T.nx) * T.ny));
        enumerate_row(T, x, y, z, m, ce);
    }
    row_len[g] = ce.count;
    const int stored = ce.count + ce.split;
    int mx = __reduce_max_sync(0xffffffffu, unsigned(stored));
    if (lane == 0) slice_len4[q] = (mx + kGroup - 1) / kGroup;
    const unsigned ns = __reduce_add_sync(0xffffffffu, unsigned(ce.split));
    if (lane == 0 && ns) atomicAdd(n_split, (unsigned long long)ns);
}

template <class VT>
__device__ __forceinline__ VT to_store(double v, float scale);
template <>
__device__ __forceinline__ double to_store<double>(double v, float) { return v; }
template <>
__device__ __forceinline__ float to_store<float>(double v, float) { return __double2float_rn(v); }

// FP16 tier: each value v is stored as one of the two FP16 numbers lo <= v /
// scale <= hi that bracket it - hi when the fraction (v/scale - lo) / (hi -
// lo) exceeds a threshold that runs through the R3 low-discrepancy sequence
// (generalised golden ratio, plastic number g: steps 1/g, 1/g^2, 1/g^3) over
// the coordinates of the column's voxel, offset per entry by a golden-ratio
// shift of (code, m).  The rounding is unbiased, deterministic, and its
// errors alternate between neighbouring source voxels, so they average out
// under the step's spreading instead of accumulating: rounding the shared
// interior stencil once (column-preserving or to nearest) leaves the same
// error in every voxel, which drifts the solution by ~1e-3 per 200 steps.
__device__ __forceinline__ double half_value(unsigned short b)
{
    return double(__half2float(__ushort_as_half(b)));
}

__device__ __forceinline__ __half round_dithered(double v, float scale, int cx, int cy, int cz, int code, int m)
{
    const double t = v / double(scale);
    const unsigned short b = __half_as_ushort(__double2half(t));
    const double hv = half_value(b);
    unsigned short lo = b, hi = b;
    if (hv > t) lo = (unsigned short)(b - 1);       // positive halves: bits are monotone
    else if (hv < t) hi = (unsigned short)(b + 1);
    if (lo == hi) return __ushort_as_half(b);
    const double a = half_value(lo), c = half_value(hi);
    const double f = (t - a) / (c - a);
    double s = code * 0.6180339887498949 + m * 0.41421356237309515;
    s -= floor(s);
    double th = cx * 0.8191725133961644 + cy * 0.671043606703789 + cz * 0.5497004779019701 + s;
    th -= floor(th);
    return __ushort_as_half(f > th ? hi : lo);
}

template <class VT>
struct FillEmit {
    VT *vals;
    uint16_t *codes;
    int64_t base;      // element index of group 0 of this lane
    float scale;
    int x, y, z, m;    // the row's voxel and direction
    int cap;           // entries the slice holds per row (count_kernel's maximum)
    int e = 0;
    __device__ void operator()(int code, double v)
    {
        if (e >= cap) return;   // count and fill enumerate the same entries; never write past the slice
        const int64_t idx = base + int64_t(e / kGroup) * (kSlice * kGroup) + (e % kGroup);
        if constexpr (std::is_same<VT, __half>::value) {
            const double t = v / double(scale);
            if (t >= kHalfSplitAt && e + 1 < cap) {
                const __half hi = __double2half(t);
                vals[idx] = hi;
                codes[idx] = uint16_t(code);
                ++e;
                const int64_t i2 = base + int64_t(e / kGroup) * (kSlice * kGroup) + (e % kGroup);
                vals[i2] = __double2half(t - double(__half2float(hi)));
                codes[i2] = uint16_t(code);
                ++e;
                return;
            }
            const int d = code / kDirs;             // source voxel = row voxel + offset d
            vals[idx] = round_dithered(v, scale, x + d % 3 - 1, y + d / 3 % 3 - 1, z + d / 9 - 1, code, m);
        } else {
            vals[idx] = to_store<VT>(v, scale);
        }
        codes[idx] = uint16_t(code);
        ++e;
    }
};

template <class VT>
__global__ void fill_kernel(DevTables T, SlicedMatrix A)
{
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t q = g / kSlice;
    const int lane = int(g % kSlice);
    if (q >= A.n_slices) return;
    const int64_t b = q / kDirs;
    const int m = int(q % kDirs);
    const int64_t v = b * kSlice + lane;
    FillEmit<VT> fe;
    fe.vals = static_cast<VT *>(A.vals);
    fe.codes = A.codes;
    fe.base = A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup;
    fe.cap = A.slice_len4[q] * kGroup;
    fe.scale = 1.0f;
    if (A.row_scale) {
        fe.scale = T.dir_scale[m];
        A.row_scale[g] = fe.scale;
    }
    if (v < T.V) {
        const int x = int(v % T.nx), y = int(v / T.nx % T.ny), z = int(v / (int64_t(T.nx) * T.ny));
        fe.x = x;
        fe.y = y;
        fe.z = z;
        fe.m = m;
        enumerate_row(T, x, y, z, m, fe);
    }
    const int total = A.slice_len4[q] * kGroup;
    for (int e = fe.e; e < total; ++e) {
        const int64_t idx = fe.base + int64_t(e / kGroup) * (kSlice * kGroup) + (e % kGroup);
        fe.vals[idx] = VT(0.0f);
        fe.codes[idx] = uint16_t(kCenterCode);
    }
}

// Column `state` = (voxel i, direction n) of the matrix built from Tf: thread
// g = d*26 + m evaluates the mass that (i, n) sends to (i + d, m), with the
// same folding as the rows (plain rows need none: there folded_contribution
// reduces to the stencil value).
__global__ void source_column_kernel(DevTables T, int64_t state, double *out)
{
    const int g = int(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= kOffs * kDirs) return;
    const int d = g / kDirs, m = g % kDirs;
    const int64_t v = state / kDirs;
    const int n = int(state % kDirs);
    const int i[3] = {int(v % T.nx), int(v / T.nx % T.ny), int(v / (int64_t(T.nx) * T.ny))};
    const int j[3] = {i[0] + d % 3 - 1, i[1] + d / 3 % 3 - 1, i[2] + d / 9 - 1};
    if (j[0] < 0 || j[1] < 0 || j[2] < 0 || j[0] >= T.nx || j[1] >= T.ny || j[2] >= T.nz) {
        out[g] = 0.0;
        return;
    }
    const int k = T.med[v];
    const int kj = T.med[vox_of(T, j[0], j[1], j[2])];
    out[g] = folded_contribution(T, i, k, __ldg(&T.nref[k]), n, j, kj, __ldg(&T.nref[kj]), m);
}

// exclusive scan of slice_len4 into slice_ptr (three passes, 1024 per block)
constexpr int kScanBlock = 1024;

__global__ void scan_blocks_kernel(const int32_t *in, int64_t n, int64_t *out, int64_t *block_sums)
{
    __shared__ int64_t s[kScanBlock];
    const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        int64_t add = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += add;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;
    if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = s[threadIdx.x];
}

__global__ void scan_sums_kernel(int64_t *block_sums, int64_t nb, int64_t *total)
{
    // single block: sequential chunks of 1024 with a running carry
    __shared__ int64_t s[kScanBlock];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        int64_t v = i < nb ? block_sums[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < kScanBlock; off <<= 1) {
            int64_t add = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
            __syncthreads();
            s[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < nb) block_sums[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry += s[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_add_kernel(int64_t *out, int64_t n, const int64_t *block_sums)
{
    const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
    if (i < n) out[i] += block_sums[blockIdx.x];
}

// canonical-order export of rows [row_begin, row_end)
__global__ void export_count_kernel(SlicedMatrix A, int64_t V, int64_t row_begin, int64_t row_end,
                                    int64_t *counts)
{
    const int64_t r = row_begin + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= row_end) return;
    const int64_t v = r / kDirs;
    const int m = int(r % kDirs);
    const int64_t g = ((v / kSlice) * kDirs + m) * kSlice + (v % kSlice);
    counts[r - row_begin] = A.row_len[g];
}

template <class VT>
__global__ void export_kernel(SlicedMatrix A, int nx, int ny, int nz, int64_t row_begin,
                              int64_t row_end, const int64_t *row_ptr, int32_t *col, double *val)
{
    const int64_t r = row_begin + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= row_end) return;
    const int64_t v = r / kDirs;
    const int m = int(r % kDirs);
    const int64_t q = (v / kSlice) * kDirs + m;
    const int lane = int(v % kSlice);
    const int64_t g = q * kSlice + lane;
    const int len = A.row_len[g];
    const int64_t base = A.slice_ptr[q] * (kSlice * kGroup) + lane * kGroup;
    const VT *vals = static_cast<const VT *>(A.vals);
    const float scale = A.row_scale ? A.row_scale[g] : 1.0f;
    const int64_t out0 = row_ptr[r - row_begin];
    int64_t out = out0;
    // FP16 split values are two consecutive entries with one code (the codes
    // of a row are otherwise distinct): add the second into the first
    const int stored = A.slice_len4[q] * kGroup;
    int prev = -1;
    for (int e = 0; e < stored; ++e) {
        const int64_t idx = base + int64_t(e / kGroup) * (kSlice * kGroup) + (e % kGroup);
        const int code = A.codes[idx];
        double x;
        if constexpr (sizeof(VT) == 2) x = double(__half2float(vals[idx])) * double(scale);
        else x = double(vals[idx]);
        if (sizeof(VT) == 2 && code == prev && out > out0) {
            val[out - 1] += x;                      // exact: two FP16 terms times a power of two
            continue;
        }
        if (out - out0 == len) break;               // padding
        const int d = code / kDirs, n = code % kDirs;
        const int64_t off = int64_t(d / 9 - 1) * nx * ny + int64_t(d / 3 % 3 - 1) * nx + (d % 3 - 1);
        col[out] = int32_t((v + off) * kDirs + n);
        val[out] = x;
        prev = code;
        ++out;
    }
}

}  // namespace

cudaError_t launch_classify(const DevTables &T, uint8_t *plain, cudaStream_t s)
{
    cudaError_t e = upload_dirs();
    if (e != cudaSuccess) return e;
    const int th = 256;
    classify_kernel<<<unsigned((T.V + th - 1) / th), th, 0, s>>>(T, plain);
    return cudaGetLastError();
}

cudaError_t launch_count(const DevTables &T, SlicedMatrix &A, unsigned long long *n_split, cudaStream_t s)
{
    cudaError_t e = upload_dirs();
    if (e != cudaSuccess) return e;
    const int th = 128;
    const int64_t rows = A.n_slices * kSlice;
    count_kernel<<<unsigned((rows + th - 1) / th), th, 0, s>>>(T, A.n_slices, A.row_len,
                                                                 A.slice_len4, n_split);
    return cudaGetLastError();
}

cudaError_t launch_scan(SlicedMatrix &A, int64_t *d_total, cudaStream_t s)
{
    const int64_t n = A.n_slices;
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    int64_t *sums = nullptr;
    cudaError_t e = cudaMallocAsync(&sums, sizeof(int64_t) * nb, s);
    if (e != cudaSuccess) return e;
    scan_blocks_kernel<<<unsigned(nb), kScanBlock, 0, s>>>(A.slice_len4, n, A.slice_ptr, sums);
    scan_sums_kernel<<<1, kScanBlock, 0, s>>>(sums, nb, d_total);
    scan_add_kernel<<<unsigned(nb), kScanBlock, 0, s>>>(A.slice_ptr, n, sums);
    e = cudaGetLastError();
    cudaError_t e2 = cudaFreeAsync(sums, s);
    return e != cudaSuccess ? e : e2;
}

cudaError_t launch_fill(const DevTables &T, SlicedMatrix &A, cudaStream_t s)
{
    const int th = 128;
    const int64_t rows = A.n_slices * kSlice;
    const unsigned blocks = unsigned((rows + th - 1) / th);
    if (A.precision == DRTS_FP64) fill_kernel<double><<<blocks, th, 0, s>>>(T, A);
    else if (A.precision == DRTS_FP32) fill_kernel<float><<<blocks, th, 0, s>>>(T, A);
    else fill_kernel<__half><<<blocks, th, 0, s>>>(T, A);
    return cudaGetLastError();
}

cudaError_t launch_source_column(const DevTables &Tf, int64_t state, double *out, cudaStream_t s)
{
    cudaError_t e = upload_dirs();
    if (e != cudaSuccess) return e;
    source_column_kernel<<<(kOffs * kDirs + 127) / 128, 128, 0, s>>>(Tf, state, out);
    return cudaGetLastError();
}

cudaError_t launch_count_export(const SlicedMatrix &A, int64_t V, int64_t row_begin,
                                int64_t row_end, int64_t *d_counts, cudaStream_t s)
{
    const int th = 256;
    const int64_t n = row_end - row_begin;
    if (n <= 0) return cudaSuccess;
    export_count_kernel<<<unsigned((n + th - 1) / th), th, 0, s>>>(A, V, row_begin, row_end, d_counts);
    return cudaGetLastError();
}

cudaError_t launch_export(const SlicedMatrix &A, int nx, int ny, int nz, int64_t row_begin,
                          int64_t row_end, const int64_t *d_row_ptr, int32_t *d_col,
                          double *d_val, cudaStream_t s)
{
    const int th = 256;
    const int64_t n = row_end - row_begin;
    if (n <= 0) return cudaSuccess;
    const unsigned blocks = unsigned((n + th - 1) / th);
    if (A.precision == DRTS_FP64)
        export_kernel<double><<<blocks, th, 0, s>>>(A, nx, ny, nz, row_begin, row_end, d_row_ptr, d_col, d_val);
    else if (A.precision == DRTS_FP32)
        export_kernel<float><<<blocks, th, 0, s>>>(A, nx, ny, nz, row_begin, row_end, d_row_ptr, d_col, d_val);
    else
        export_kernel<__half><<<blocks, th, 0, s>>>(A, nx, ny, nz, row_begin, row_end, d_row_ptr, d_col, d_val);
    return cudaGetLastError();
}

}  // namespace drts
