// The DRTS step of Eq. 26, x(t+1) = A x(t) + s(t), on the close-packed sphere
// partition of Section 3 (face-centred cubic sites, 12 nearest-neighbour
// directions), with A (Eq. 18-21, 23) assembled on the device.
//
// Sites are integer triples (i, j, k) with i + j + k even; site index
// v = ((k ny + j) nx + i) / 2, so the nx / 2 sites of a lattice row (j, k)
// share the parity p = (j + k) mod 2 of their x coordinates (i = 2h + p).
// The source of lattice offset (dx, dy, dz) for target site v is the site
//     v - dz ny nx/2 - dy nx/2 + floor((p - dx) / 2),
// so the column of an entry is fixed by its code (offset o, direction n) and
// the row's parity: two code -> column tables, selected per lane.
//
// Layout (as on the voxel grid): slice q = b * 12 + m holds the rows
// (site 32 b + l, direction m), l = 0..31; entry e of lane l sits at
// ((slice_ptr[q] + e / 4) * 32 + l) * 4 + e % 4 (a lane moves 4 consecutive
// entries per load); rows are padded to the slice's longest row rounded to
// 4 with value 0 and the code of the site itself.  State: direction-major,
// x[d * S + v], S = n_sites + 64 (the tail keeps the padding lanes of the
// last slice in bounds and stays zero).
//
// Assembly: the host evaluates each medium's stencil in FP64 (transition
// weights by offset and direction pair, the only transcendental work); the
// device counts every row (the sources inside the box, their media and the
// nonzero weights), scans the slice lengths and fills the rows in ascending
// column order (offsets sorted by their site delta for the row's parity,
// then source direction).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "drts_device.cuh"
#include "drts_internal.h"

namespace drts {
namespace {

constexpr int kMaxFccOff = 64;                      // offsets the shared-memory tables hold
constexpr int kFccCodes = kMaxFccOff * kFccDirs;    // 768 codes
constexpr int kFccMaxSrc = 64;

struct FccGeom {
    int nx, ny, nz;
    int half;               // nx / 2 sites per lattice row
    int64_t n_sites;
    int64_t S;              // state stride of one direction
    int n_off;
    int K;                  // media
};

// lattice coordinates of site v
__device__ __forceinline__ void fcc_coords(const FccGeom &g, int64_t v, int &i, int &j, int &k)
{
    const int64_t row = v / g.half;
    const int h = int(v - row * g.half);
    j = int(row % g.ny);
    k = int(row / g.ny);
    i = 2 * h + ((j + k) & 1);
}

// The source of offset o for target (i, j, k) inside the box, or -1.
__device__ __forceinline__ int64_t fcc_source(const FccGeom &g, const int *off3, int o, int i, int j, int k)
{
    const int si = i - off3[3 * o], sj = j - off3[3 * o + 1], sk = k - off3[3 * o + 2];
    if (si < 0 || si >= g.nx || sj < 0 || sj >= g.ny || sk < 0 || sk >= g.nz) return -1;
    return ((int64_t(sk) * g.ny + sj) * g.nx + si) / 2;
}

// Row lengths (one warp per slice, one lane per row) and slice lengths in
// groups of 4 entries.
__global__ void fcc_count_kernel(FccGeom g, const int *off3, const double *W, const uint8_t *med,
                                 int64_t n_slices, int32_t *row_len, int32_t *slice_len4)
{
    const int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= n_slices) return;                       // whole warps leave together
    const int64_t v = (q / kFccDirs) * 32 + lane;
    const int m = int(q % kFccDirs);
    int cnt = 0;
    if (v < g.n_sites) {
        int i, j, k;
        fcc_coords(g, v, i, j, k);
        for (int o = 0; o < g.n_off; ++o) {
            const int64_t src = fcc_source(g, off3, o, i, j, k);
            if (src < 0) continue;
            const double *w = W + ((size_t(med[src]) * g.n_off + o) * kFccDirs) * kFccDirs + m;
            for (int n = 0; n < kFccDirs; ++n) cnt += w[n * kFccDirs] > 0.0;
        }
    }
    row_len[q * 32 + lane] = cnt;
    const int mx = __reduce_max_sync(0xffffffffu, cnt);
    if (lane == 0) slice_len4[q] = (mx + 3) / 4;
}

// Entries of every row in ascending column order: the row's parity picks
// the offset order (ascending site delta), then the source direction.
template <class T>
__global__ void fcc_fill_kernel(FccGeom g, const int *off3, const int *ord, const double *W, const uint8_t *med,
                                int64_t n_slices, const int64_t *slice_ptr, const int32_t *slice_len4, T *vals,
                                uint16_t *codes)
{
    const int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= n_slices) return;
    const int64_t v = (q / kFccDirs) * 32 + lane;
    const int m = int(q % kFccDirs);
    const int64_t base = slice_ptr[q];
    const int cap = 4 * slice_len4[q];
    int e = 0;
    auto put = [&](T val, int code) {
        const int64_t idx = ((base + e / 4) * 32 + lane) * 4 + e % 4;
        vals[idx] = val;
        codes[idx] = uint16_t(code);
        ++e;
    };
    if (v < g.n_sites) {
        int i, j, k;
        fcc_coords(g, v, i, j, k);
        const int *order = ord + ((j + k) & 1) * g.n_off;
        for (int oo = 0; oo < g.n_off; ++oo) {
            const int o = order[oo];
            const int64_t src = fcc_source(g, off3, o, i, j, k);
            if (src < 0) continue;
            const double *w = W + ((size_t(med[src]) * g.n_off + o) * kFccDirs) * kFccDirs + m;
            for (int n = 0; n < kFccDirs; ++n)
                if (w[n * kFccDirs] > 0.0 && e < cap) put(T(w[n * kFccDirs]), o * kFccDirs + n);
        }
    }
    while (e < cap) put(T(0), 0);                    // offset 0 is the site itself, direction 0
}

// One step y = A x: one warp per slice, one lane per row; codes map to
// column offsets through the shared-memory table of the row's parity
// (tab[p][o * 12 + n] = n S + site delta).  FP64 or FP32 accumulation in
// entry order.
template <class T>
__global__ void __launch_bounds__(256) fcc_step_kernel(FccGeom g, int64_t n_slices, const int64_t *slice_ptr,
                                                       const int32_t *slice_len4, const T *vals,
                                                       const uint16_t *codes, const int32_t *coltab, const T *x,
                                                       T *y)
{
    __shared__ int32_t tab[2][kFccCodes];
    for (int c = threadIdx.x; c < 2 * g.n_off * kFccDirs; c += blockDim.x) {
        const int p = c / (g.n_off * kFccDirs), r = c % (g.n_off * kFccDirs);
        tab[p][r] = coltab[c];
    }
    __syncthreads();
    const int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= n_slices) return;
    const int64_t v = (q / kFccDirs) * 32 + lane;
    const int m = int(q % kFccDirs);
    const int p = v < g.n_sites ? int(((v / g.half) % g.ny + (v / g.half) / g.ny) & 1) : 0;
    const int32_t *tp = tab[p];
    const int64_t base = slice_ptr[q];
    const int len4 = slice_len4[q];
    T acc = T(0);
    for (int gi = 0; gi < len4; ++gi) {
        const int64_t idx = ((base + gi) * 32 + lane) * 4;
        const uint2 cw = *reinterpret_cast<const uint2 *>(codes + idx);
        T w[4];
        if constexpr (sizeof(T) == 4) {
            const float4 f = *reinterpret_cast<const float4 *>(vals + idx);
            w[0] = f.x; w[1] = f.y; w[2] = f.z; w[3] = f.w;
        } else {
            const double2 a = *reinterpret_cast<const double2 *>(vals + idx);
            const double2 b = *reinterpret_cast<const double2 *>(vals + idx + 2);
            w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
        }
        const uint32_t c4[4] = {cw.x & 0xFFFFu, cw.x >> 16, cw.y & 0xFFFFu, cw.y >> 16};
#pragma unroll
        for (int u = 0; u < 4; ++u) acc += w[u] * x[v + tp[c4[u]]];
    }
    if (v < g.n_sites) y[int64_t(m) * g.S + v] = acc;
}

// s(t) of Eq. 26: y[state] += weight * P(t)
template <class T>
__global__ void fcc_source_kernel(FccGeom g, int n, const int64_t *states, const double *weights, double scale, T *y)
{
    const int e = threadIdx.x;
    if (e >= n) return;
    const int64_t st = states[e];
    const int64_t v = st / kFccDirs;
    const int d = int(st % kFccDirs);
    y[int64_t(d) * g.S + v] += T(weights[e] * scale);   // distinct states: no two threads share a target
}

template <class T>
__global__ void fcc_to_states_kernel(FccGeom g, const T *x, double *out)
{
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= g.n_sites * kFccDirs) return;
    out[r] = double(x[(r % kFccDirs) * g.S + r / kFccDirs]);
}

// Row lengths of rows [r0, r1) in state order (row v * 12 + m)
__global__ void fcc_export_len_kernel(int64_t r0, int64_t r1, const int32_t *row_len, int64_t *out)
{
    const int64_t r = r0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= r1) return;
    const int64_t v = r / kFccDirs;
    const int m = int(r % kFccDirs);
    out[r - r0] = row_len[((v / 32) * kFccDirs + m) * 32 + v % 32];
}

template <class T>
__global__ void fcc_export_kernel(FccGeom g, int64_t r0, int64_t r1, const int64_t *rp, const int32_t *row_len,
                                  const int64_t *slice_ptr, const T *vals, const uint16_t *codes,
                                  const int32_t *coltab, int32_t *col, double *val)
{
    const int64_t r = r0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= r1) return;
    const int64_t v = r / kFccDirs;
    const int m = int(r % kFccDirs);
    const int64_t q = (v / 32) * kFccDirs + m;
    const int lane = int(v % 32);
    const int len = row_len[q * 32 + lane];
    const int p = int(((v / g.half) % g.ny + (v / g.half) / g.ny) & 1);
    int64_t out = rp[r - r0];
    for (int e = 0; e < len; ++e, ++out) {
        const int64_t idx = ((slice_ptr[q] + e / 4) * 32 + lane) * 4 + e % 4;
        const int code = codes[idx];
        // column of the entry: direction n of site v + delta
        const int n = code % kFccDirs;
        const int64_t src = v + (coltab[p * g.n_off * kFccDirs + code] - int64_t(n) * g.S);
        col[out] = int32_t(src * kFccDirs + n);
        val[out] = double(vals[idx]);
    }
}

}  // namespace
}  // namespace drts

using namespace drts;

struct drts_fcc_ctx {
    cudaStream_t stream = nullptr;
    int precision = DRTS_FP32;
    FccGeom g{};
    SlicedMatrix A;                  // vals, codes, slice_ptr, slice_len4, row_len
    int32_t *coltab = nullptr;       // [2][n_off * 12]
    void *x = nullptr, *y = nullptr; // [12 * S] each
    int64_t *src_states = nullptr;   // [kFccMaxSrc]
    double *src_w = nullptr;
    int n_src = 0;
    int64_t t0 = 0;
    std::vector<double> profile;
    int64_t t = 0;
    std::vector<void *> allocs;
};

namespace {

drts_status fcc_err(drts_status s, const std::string &m)
{
    set_global_error(m);
    return s;
}

drts_status fcc_cuda(cudaError_t e, const char *where)
{
    cudaGetLastError();
    return fcc_err(e == cudaErrorMemoryAllocation ? DRTS_ENOMEM : DRTS_ECUDA,
                   std::string(where) + ": " + cudaGetErrorString(e));
}

template <class T>
cudaError_t fcc_alloc(drts_fcc_ctx *c, T **p, size_t bytes)
{
    void *q = nullptr;
    const cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return cudaSuccess;
}

void fcc_free(drts_fcc_ctx *c)
{
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (void *p : c->allocs) cudaFree(p);
    c->allocs.clear();
}

template <class T>
cudaError_t fcc_launch_step(drts_fcc_ctx *c)
{
    const int64_t warps = c->A.n_slices;
    const unsigned blocks = unsigned((warps + 7) / 8);
    fcc_step_kernel<T><<<blocks, 256, 0, c->stream>>>(c->g, c->A.n_slices, c->A.slice_ptr, c->A.slice_len4,
                                                      static_cast<const T *>(c->A.vals), c->A.codes, c->coltab,
                                                      static_cast<const T *>(c->x), static_cast<T *>(c->y));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (c->n_src > 0 && c->t >= c->t0 && c->t < c->t0 + int64_t(c->profile.size())) {
        const double scale = c->profile[size_t(c->t - c->t0)];
        fcc_source_kernel<T><<<1, kFccMaxSrc, 0, c->stream>>>(c->g, c->n_src, c->src_states, c->src_w, scale,
                                                             static_cast<T *>(c->y));
        e = cudaGetLastError();
    }
    std::swap(c->x, c->y);
    ++c->t;
    return e;
}

}  // namespace

extern "C" {

drts_status drts_fcc_assemble(const drts_fcc_problem *prob, int32_t precision, void *cuda_stream,
                              drts_fcc_ctx **out)
try {
    NvtxRange nvtx("drts_fcc_assemble");
    if (!out) return fcc_err(DRTS_EINVAL, "out is NULL");
    *out = nullptr;
    drts_status st = fcc_validate(prob);
    if (st != DRTS_OK) return st;
    if (precision != DRTS_FP64 && precision != DRTS_FP32)
        return fcc_err(DRTS_EUNSUPPORTED, "the close-packed step supports DRTS_FP64 and DRTS_FP32");
    FccTables T;
    fcc_tables(*prob, T);
    const int n_off = int(T.off.size());
    if (n_off > kMaxFccOff) return fcc_err(DRTS_EUNSUPPORTED, "stencil reaches more lattice offsets than the tables hold");
    drts_fcc_ctx *c = new drts_fcc_ctx;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->precision = precision;
    FccGeom &g = c->g;
    g.nx = prob->nx;
    g.ny = prob->ny;
    g.nz = prob->nz;
    g.half = prob->nx / 2;
    g.n_sites = int64_t(prob->nx) * prob->ny * prob->nz / 2;
    g.S = g.n_sites + 64;
    g.n_off = n_off;
    g.K = prob->n_media;
    // per parity: site delta of each offset, the offsets by ascending delta,
    // and the code -> column-offset table of the step
    std::vector<int> off3(size_t(3 * n_off)), ord(size_t(2 * n_off));
    std::vector<int32_t> coltab(size_t(2 * n_off * kFccDirs));
    for (int p = 0; p < 2; ++p) {
        std::vector<std::pair<int64_t, int>> by;
        for (int o = 0; o < n_off; ++o) {
            const int dx = T.off[size_t(o)][0], dy = T.off[size_t(o)][1], dz = T.off[size_t(o)][2];
            const int fl = (p - dx) >= 0 ? (p - dx) / 2 : -((dx - p + 1) / 2);   // floor((p - dx) / 2)
            const int64_t delta = -int64_t(dz) * g.ny * g.half - int64_t(dy) * g.half + fl;
            by.emplace_back(delta, o);
            for (int n = 0; n < kFccDirs; ++n)
                coltab[size_t((p * n_off + o) * kFccDirs + n)] = int32_t(int64_t(n) * g.S + delta);
            if (p == 0) {
                off3[size_t(3 * o)] = dx;
                off3[size_t(3 * o + 1)] = dy;
                off3[size_t(3 * o + 2)] = dz;
            }
        }
        std::stable_sort(by.begin(), by.end());
        for (int o = 0; o < n_off; ++o) ord[size_t(p * n_off + o)] = by[size_t(o)].second;
    }
    const int64_t n_slices = (g.n_sites + 31) / 32 * kFccDirs;
    int *d_off3 = nullptr, *d_ord = nullptr;
    double *d_W = nullptr;
    uint8_t *d_med = nullptr;
    int64_t *d_total = nullptr;
    cudaError_t e;
    auto fail = [&](cudaError_t err, const char *where) {
        const drts_status s2 = fcc_cuda(err, where);
        fcc_free(c);
        delete c;
        return s2;
    };
    if ((e = fcc_alloc(c, &d_off3, off3.size() * sizeof(int))) != cudaSuccess ||
        (e = fcc_alloc(c, &d_ord, ord.size() * sizeof(int))) != cudaSuccess ||
        (e = fcc_alloc(c, &d_W, T.W.size() * sizeof(double))) != cudaSuccess ||
        (e = fcc_alloc(c, &d_med, size_t(g.n_sites))) != cudaSuccess ||
        (e = fcc_alloc(c, &c->coltab, coltab.size() * sizeof(int32_t))) != cudaSuccess ||
        (e = fcc_alloc(c, &d_total, sizeof(int64_t))) != cudaSuccess ||
        (e = fcc_alloc(c, &c->A.row_len, size_t(n_slices) * 32 * sizeof(int32_t))) != cudaSuccess ||
        (e = fcc_alloc(c, &c->A.slice_len4, size_t(n_slices) * sizeof(int32_t))) != cudaSuccess ||
        (e = fcc_alloc(c, &c->A.slice_ptr, size_t(n_slices) * sizeof(int64_t))) != cudaSuccess ||
        (e = fcc_alloc(c, &c->src_states, kFccMaxSrc * sizeof(int64_t))) != cudaSuccess ||
        (e = fcc_alloc(c, &c->src_w, kFccMaxSrc * sizeof(double))) != cudaSuccess)
        return fail(e, "close-packed table allocation");
    if ((e = cudaMemcpyAsync(d_off3, off3.data(), off3.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(d_ord, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(d_W, T.W.data(), T.W.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(d_med, prob->medium_of_site, size_t(g.n_sites), cudaMemcpyHostToDevice, c->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(c->coltab, coltab.data(), coltab.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess)
        return fail(e, "close-packed table upload");
    c->A.precision = precision;
    c->A.n_slices = n_slices;
    const unsigned blocks = unsigned((n_slices * 32 + 127) / 128);
    fcc_count_kernel<<<blocks, 128, 0, c->stream>>>(g, d_off3, d_W, d_med, n_slices, c->A.row_len, c->A.slice_len4);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = launch_scan(c->A, d_total, c->stream)) != cudaSuccess)
        return fail(e, "close-packed row count");
    int64_t groups = 0;
    if ((e = cudaMemcpyAsync(&groups, d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return fail(e, "close-packed row count");
    c->A.n_groups = groups;
    const size_t slots = size_t(groups) * 128;
    const size_t vb = precision == DRTS_FP64 ? 8 : 4;
    if ((e = fcc_alloc(c, &c->A.vals, slots * vb)) != cudaSuccess ||
        (e = fcc_alloc(c, &c->A.codes, slots * sizeof(uint16_t))) != cudaSuccess ||
        (e = fcc_alloc(c, &c->x, size_t(kFccDirs) * size_t(g.S) * vb)) != cudaSuccess ||
        (e = fcc_alloc(c, &c->y, size_t(kFccDirs) * size_t(g.S) * vb)) != cudaSuccess)
        return fail(e, "close-packed matrix allocation");
    if ((e = cudaMemsetAsync(c->x, 0, size_t(kFccDirs) * size_t(g.S) * vb, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->y, 0, size_t(kFccDirs) * size_t(g.S) * vb, c->stream)) != cudaSuccess)
        return fail(e, "close-packed state");
    if (precision == DRTS_FP64)
        fcc_fill_kernel<double><<<blocks, 128, 0, c->stream>>>(g, d_off3, d_ord, d_W, d_med, n_slices, c->A.slice_ptr,
                                                              c->A.slice_len4, static_cast<double *>(c->A.vals),
                                                              c->A.codes);
    else
        fcc_fill_kernel<float><<<blocks, 128, 0, c->stream>>>(g, d_off3, d_ord, d_W, d_med, n_slices, c->A.slice_ptr,
                                                             c->A.slice_len4, static_cast<float *>(c->A.vals),
                                                             c->A.codes);
    // the row lengths' sum is the stored nonzero count
    std::vector<int32_t> lens(size_t(n_slices) * 32);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(lens.data(), c->A.row_len, lens.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                             c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return fail(e, "close-packed fill");
    int64_t nnz = 0;
    for (int32_t l : lens) nnz += l;
    c->A.nnz = c->A.nnz_stored = nnz;
    *out = c;
    return DRTS_OK;
} catch (const std::bad_alloc &) {
    return fcc_err(DRTS_ENOMEM, "drts_fcc_assemble: host allocation failed");
} catch (...) {
    return fcc_err(DRTS_EINVAL, "drts_fcc_assemble: unexpected exception");
}

drts_status drts_fcc_set_source(drts_fcc_ctx *c, int32_t n, const int64_t *states, const double *weights,
                                int64_t t0, int32_t n_t, const double *profile)
try {
    if (!c) return fcc_err(DRTS_EINVAL, "context is NULL");
    if (n < 0 || n > kFccMaxSrc || (n > 0 && (!states || !weights))) return fcc_err(DRTS_EINVAL, "0..64 source states");
    if (n_t < 0 || (n_t > 0 && !profile)) return fcc_err(DRTS_EINVAL, "bad profile");
    const int64_t ns = c->g.n_sites * kFccDirs;
    for (int i = 0; i < n; ++i) {
        if (states[i] < 0 || states[i] >= ns) return fcc_err(DRTS_EINVAL, "source state out of range");
        for (int k = 0; k < i; ++k)
            if (states[k] == states[i]) return fcc_err(DRTS_EINVAL, "repeated source state");
    }
    cudaError_t e;
    if (n > 0 &&
        ((e = cudaMemcpyAsync(c->src_states, states, size_t(n) * sizeof(int64_t), cudaMemcpyHostToDevice,
                              c->stream)) != cudaSuccess ||
         (e = cudaMemcpyAsync(c->src_w, weights, size_t(n) * sizeof(double), cudaMemcpyHostToDevice, c->stream)) !=
             cudaSuccess ||
         (e = cudaStreamSynchronize(c->stream)) != cudaSuccess))
        return fcc_cuda(e, "close-packed source upload");
    c->n_src = n;
    c->t0 = t0;
    c->profile.assign(profile, profile + n_t);
    return DRTS_OK;
} catch (...) {
    return fcc_err(DRTS_ENOMEM, "drts_fcc_set_source: host allocation failed");
}

drts_status drts_fcc_step_n(drts_fcc_ctx *c, int64_t n)
try {
    if (!c) return fcc_err(DRTS_EINVAL, "context is NULL");
    if (n < 0) return fcc_err(DRTS_EINVAL, "n must be >= 0");
    NvtxRange nvtx("drts_fcc_step_n");
    for (int64_t s = 0; s < n; ++s) {
        const cudaError_t e = c->precision == DRTS_FP64 ? fcc_launch_step<double>(c) : fcc_launch_step<float>(c);
        if (e != cudaSuccess) return fcc_cuda(e, "close-packed step");
    }
    return DRTS_OK;
} catch (...) {
    return fcc_err(DRTS_EINVAL, "drts_fcc_step_n: unexpected exception");
}

drts_status drts_fcc_read_state(drts_fcc_ctx *c, double *host_out)
try {
    if (!c || !host_out) return fcc_err(DRTS_EINVAL, "context or output is NULL");
    const int64_t ns = c->g.n_sites * kFccDirs;
    double *d = nullptr;
    cudaError_t e = cudaMallocAsync(&d, size_t(ns) * sizeof(double), c->stream);
    if (e != cudaSuccess) return fcc_cuda(e, "close-packed read_state");
    const unsigned blocks = unsigned((ns + 255) / 256);
    if (c->precision == DRTS_FP64)
        fcc_to_states_kernel<double><<<blocks, 256, 0, c->stream>>>(c->g, static_cast<const double *>(c->x), d);
    else
        fcc_to_states_kernel<float><<<blocks, 256, 0, c->stream>>>(c->g, static_cast<const float *>(c->x), d);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, d, size_t(ns) * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    const cudaError_t e2 = cudaFreeAsync(d, c->stream);
    const cudaError_t e3 = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
    return e == cudaSuccess ? DRTS_OK : fcc_cuda(e, "close-packed read_state");
} catch (...) {
    return fcc_err(DRTS_EINVAL, "drts_fcc_read_state: unexpected exception");
}

drts_status drts_fcc_read_rows(drts_fcc_ctx *c, int64_t r0, int64_t r1, int64_t *row_ptr, int32_t *col, double *val,
                               int64_t cap)
try {
    if (!c || !row_ptr) return fcc_err(DRTS_EINVAL, "context or row_ptr is NULL");
    const int64_t ns = c->g.n_sites * kFccDirs;
    if (r0 < 0 || r1 < r0 || r1 > ns) return fcc_err(DRTS_EINVAL, "bad row range");
    const int64_t nr = r1 - r0;
    int64_t *d_len = nullptr, *d_rp = nullptr;
    int32_t *d_col = nullptr;
    double *d_val = nullptr;
    std::vector<int64_t> lens(static_cast<size_t>(nr));
    cudaError_t e = cudaMallocAsync(&d_len, size_t(nr + 1) * sizeof(int64_t), c->stream);
    if (e != cudaSuccess) return fcc_cuda(e, "close-packed read_rows");
    const unsigned blocks = unsigned((nr + 255) / 256);
    if (nr > 0) fcc_export_len_kernel<<<blocks, 256, 0, c->stream>>>(r0, r1, c->A.row_len, d_len);
    e = cudaGetLastError();
    if (e == cudaSuccess && nr > 0)
        e = cudaMemcpyAsync(lens.data(), d_len, size_t(nr) * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(d_len, c->stream);
        return fcc_cuda(e, "close-packed read_rows");
    }
    row_ptr[0] = 0;
    for (int64_t r = 0; r < nr; ++r) row_ptr[r + 1] = row_ptr[r] + lens[size_t(r)];
    const int64_t total = row_ptr[nr];
    if (total > cap || (total > 0 && (!col || !val))) {
        cudaFreeAsync(d_len, c->stream);
        cudaStreamSynchronize(c->stream);
        return fcc_err(DRTS_EINVAL, "capacity " + std::to_string(cap) + " < " + std::to_string(total) + " entries");
    }
    d_rp = d_len;                      // reused for the row pointers
    if ((e = cudaMemcpyAsync(d_rp, row_ptr, size_t(nr + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream)) ==
            cudaSuccess &&
        (e = cudaMallocAsync(&d_col, size_t(total + 1) * sizeof(int32_t), c->stream)) == cudaSuccess &&
        (e = cudaMallocAsync(&d_val, size_t(total + 1) * sizeof(double), c->stream)) == cudaSuccess) {
        if (nr > 0) {
            if (c->precision == DRTS_FP64)
                fcc_export_kernel<double><<<blocks, 256, 0, c->stream>>>(
                    c->g, r0, r1, d_rp, c->A.row_len, c->A.slice_ptr, static_cast<const double *>(c->A.vals),
                    c->A.codes, c->coltab, d_col, d_val);
            else
                fcc_export_kernel<float><<<blocks, 256, 0, c->stream>>>(
                    c->g, r0, r1, d_rp, c->A.row_len, c->A.slice_ptr, static_cast<const float *>(c->A.vals),
                    c->A.codes, c->coltab, d_col, d_val);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && total > 0)
            e = cudaMemcpyAsync(col, d_col, size_t(total) * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && total > 0)
            e = cudaMemcpyAsync(val, d_val, size_t(total) * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    }
    if (d_col) cudaFreeAsync(d_col, c->stream);
    if (d_val) cudaFreeAsync(d_val, c->stream);
    cudaFreeAsync(d_len, c->stream);
    const cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = e2;
    return e == cudaSuccess ? DRTS_OK : fcc_cuda(e, "close-packed read_rows");
} catch (...) {
    return fcc_err(DRTS_EINVAL, "drts_fcc_read_rows: unexpected exception");
}

drts_status drts_fcc_get_info(const drts_fcc_ctx *c, drts_fcc_info *out)
{
    if (!c || !out) return fcc_err(DRTS_EINVAL, "context or output is NULL");
    std::memset(out, 0, sizeof(*out));
    out->n_sites = c->g.n_sites;
    out->n_states = c->g.n_sites * kFccDirs;
    out->nnz = c->A.nnz;
    out->slots = c->A.n_groups * 128;
    out->n_offsets = c->g.n_off;
    out->precision = c->precision;
    out->t = c->t;
    out->matrix_bytes = out->slots * ((c->precision == DRTS_FP64 ? 8 : 4) + 2);
    return DRTS_OK;
}

drts_status drts_fcc_destroy(drts_fcc_ctx *c)
{
    if (!c) return DRTS_OK;
    fcc_free(c);
    delete c;
    return DRTS_OK;
}

}  // extern "C"
