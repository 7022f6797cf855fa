// C ABI of libdrts (declared in include/drts.h): context life cycle,
// assembly, sources, stepping, readout.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <exception>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "drts_device.cuh"

using namespace drts;

namespace {
// The device allocator of context buffers (drts_set_allocator); null
// functions mean cudaMalloc / cudaFree.
struct Allocator {
    drts_alloc_fn alloc = nullptr;
    drts_free_fn free = nullptr;
    void *user = nullptr;
};
// a context buffer and the allocator that owns it
struct DevBuffer {
    void *p = nullptr;
    Allocator a;
};
}  // namespace

struct drts_ctx {
    drts_problem prob{};
    cudaStream_t stream = nullptr;
    int64_t V = 0, n_states = 0;
    int K = 0, R = 1, n_patch = 0;
    int64_t rhs_stride = 0;              // elements between right-hand sides of a state buffer
    bool tc = false;                     // tensor-core batched step (8 KB bf16 state tile per voxel)
    TcPlan tcp{};                        // its union-dense A
    uint8_t *d_src_voxel = nullptr;      // [V] voxels that receive a source term
    int64_t t = 0;
    std::string err;
    HostTables host;
    DevTables T{};
    SlicedMatrix A{};
    // device buffers
    std::vector<DevBuffer> allocs;
    void *x = nullptr, *y = nullptr;     // state ping-pong
    int64_t x_elems = 0;
    double *ledger = nullptr;            // [R][4]
    double *det = nullptr;               // [R][max_steps][n_patch]
    double *d_absorb = nullptr, *d_exit_tot = nullptr, *d_exit_det = nullptr;   // per ledger class
    double *d_absorb_dir = nullptr;      // [C][26] two-step interfaces, else null
    uint8_t *d_cls = nullptr;            // [V] ledger class of each voxel (= d_med without two-step)
    std::vector<uint8_t> cls_host;       // [V] host copy (two-step interfaces only; else med_host)
    SourceEntry *d_src = nullptr;
    SourceProfile *d_prof = nullptr;
    double *d_prof_vals = nullptr;
    int64_t prof_cap = 0;
    std::vector<SourceEntry> src;        // host copy of all rhs entries
    std::vector<SourceProfile> prof;     // [R]
    std::vector<std::vector<double>> prof_vals;
    int blocks = 0, threads = 256, rhs_tile = 0, variant = 0;
    int *d_err = nullptr;                // device error word of bounded waits
    uint32_t spin_limit = 1u << 22;
    int64_t fault_skip_chunk = -1;
    int fault_skip_barrier = 0;
    int step_mode = DRTS_STEP_LAUNCH;
    unsigned *d_bar = nullptr;           // grid barrier of the persistent kernel
    int special_permille = 0;
    std::vector<drts_medium> media;      // the problem's media (partial-path tables)
    uint8_t *d_med = nullptr;            // [V] medium of each voxel (device)
    std::vector<uint8_t> med_host;       // [V] medium of each voxel (host copy)
    // point detectors (sparse detector rows F of Eq. 27)
    int n_pdet = 0;
    int64_t *d_pdet_off = nullptr, *d_pdet_state = nullptr;
    double *d_pdet_w = nullptr, *d_pdet_hist = nullptr;
    // sub-step sources, per rhs: entries (state, weight), n_sub, t0, n_t, profile [n_t][n_sub]
    struct SubstepSource {
        std::vector<int64_t> state;
        std::vector<double> weight;
        int n_sub = 0;
        int64_t t0 = 0;
        int32_t n_t = 0;
        std::vector<double> profile;
        std::vector<std::vector<std::pair<int64_t, double>>> columns;   // [entry * n_sub + j]
    };
    std::vector<SubstepSource> substep;  // [R]
    int n_bulk_groups = 0;
    BulkGroup *d_bulk_groups = nullptr;
    int32_t *d_bulk_rhs_off = nullptr;
    BulkEntry *d_bulk_entries = nullptr;
    SourceProfile *d_bulk_prof = nullptr;
    double *d_bulk_prof_vals = nullptr;
};

namespace {

// message of the last failed context-free call (drts_assemble and the
// diagnostics) on this thread
thread_local std::string g_assemble_error;

drts_status fail(drts_ctx *c, drts_status s, const std::string &msg)
{
    if (c) c->err = msg;
    else g_assemble_error = msg;
    return s;
}

// No C++ exception may cross the C ABI: each entry point's handler turns the
// one in flight into a status (a failed host allocation is DRTS_ENOMEM,
// anything else DRTS_EINVAL) and records the message.  Call only from a catch
// handler.
drts_status caught(drts_ctx *c, const char *where) noexcept
{
    drts_status st = DRTS_EINVAL;
    const char *what = "unknown exception";
    try {
        throw;
    } catch (const std::bad_alloc &) {
        st = DRTS_ENOMEM;
        what = "host allocation failed";
    } catch (const std::exception &ex) {
        what = ex.what();
    } catch (...) {
    }
    try {
        fail(c, st, std::string(where) + ": " + what);
    } catch (...) {
    }
    return st;
}

drts_status cuda_fail(drts_ctx *c, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? DRTS_ENOMEM : DRTS_ECUDA, m);
}

// Allocator fault for tests (drts_set_alloc_fault): successful context
// allocations left before one fails; negative = disarmed.
std::atomic<int64_t> g_alloc_fault{-1};

bool alloc_fault_fires()
{
    int64_t n = g_alloc_fault.load();
    while (n >= 0) {
        // n > 0: one more allocation may succeed; n == 0: this one fails and
        // the fault disarms itself
        if (g_alloc_fault.compare_exchange_weak(n, n > 0 ? n - 1 : -1)) return n == 0;
    }
    return false;
}

std::mutex g_allocator_mu;
Allocator g_allocator;

Allocator current_allocator()
{
    std::lock_guard<std::mutex> lock(g_allocator_mu);
    return g_allocator;
}

void free_buffer(const DevBuffer &b, cudaStream_t s)
{
    if (b.a.free) b.a.free(b.p, s, b.a.user);
    else cudaFree(b.p);
}

template <class T>
cudaError_t dalloc(drts_ctx *c, T **p, size_t bytes)
{
    void *q = nullptr;
    if (alloc_fault_fires()) return cudaErrorMemoryAllocation;
    const Allocator a = current_allocator();
    cudaError_t e = cudaSuccess;
    if (a.alloc) {
        q = a.alloc(bytes ? bytes : 16, c->stream, a.user);
        if (!q) return cudaErrorMemoryAllocation;
        if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {     // bulk copies and vector loads need it
            a.free(q, c->stream, a.user);
            return cudaErrorMisalignedAddress;
        }
    } else {
        e = cudaMalloc(&q, bytes ? bytes : 16);
    }
    if (e == cudaSuccess) {
        c->allocs.push_back(DevBuffer{q, a});
        *p = static_cast<T *>(q);
    }
    return e;
}

// Free a buffer from dalloc and forget it (the context stream is drained
// first: kernels already queued may still read it).  No-op on NULL.
template <class T>
void drelease(drts_ctx *c, T *&p)
{
    if (!p) return;
    cudaStreamSynchronize(c->stream);
    auto it = std::find_if(c->allocs.begin(), c->allocs.end(),
                           [&](const DevBuffer &b) { return b.p == static_cast<void *>(p); });
    if (it != c->allocs.end()) {
        const DevBuffer b = *it;
        c->allocs.erase(it);
        free_buffer(b, c->stream);
    }
    p = nullptr;
}

template <class T>
cudaError_t upload(drts_ctx *c, T **p, const std::vector<T> &v)
{
    cudaError_t e = dalloc(c, p, v.size() * sizeof(T));
    if (e == cudaSuccess && !v.empty())
        e = cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream);
    return e;
}

size_t state_elem_bytes(int precision) { return precision == DRTS_FP64 ? 8 : 4; }

size_t value_bytes(int precision) { return precision == DRTS_FP64 ? 8 : (precision == DRTS_FP32 ? 4 : 2); }

drts_status validate(const drts_problem *p)
{
    if (!p) return fail(nullptr, DRTS_EINVAL, "problem is NULL");
    if (p->nx < 2 || p->ny < 2 || p->nz < 2) return fail(nullptr, DRTS_EINVAL, "grid sides must be >= 2");
    const int64_t V = int64_t(p->nx) * p->ny * p->nz;
    if (V * kDirs >= (int64_t(1) << 31)) return fail(nullptr, DRTS_EINVAL, "more than 2^31 states");
    if (!(p->voxel_mm > 0.0)) return fail(nullptr, DRTS_EINVAL, "voxel_mm must be > 0");
    if (p->n_media < 1 || p->n_media > 255 || !p->media) return fail(nullptr, DRTS_EINVAL, "n_media must be 1..255");
    if (!p->medium_of_voxel) return fail(nullptr, DRTS_EINVAL, "medium_of_voxel is NULL");
    for (int k = 0; k < p->n_media; ++k) {
        const drts_medium &m = p->media[k];
        if (!(m.n > 0.0) || m.mu_s < 0.0 || m.mu_a < 0.0 || !(m.g > -1.0 && m.g < 1.0))
            return fail(nullptr, DRTS_EINVAL, "medium " + std::to_string(k) + " out of range");
    }
    for (int64_t v = 0; v < V; ++v)
        if (p->medium_of_voxel[v] >= p->n_media) return fail(nullptr, DRTS_EINVAL, "medium index out of range");
    if (p->boundary < DRTS_OPEN || p->boundary > DRTS_FRESNEL) return fail(nullptr, DRTS_EINVAL, "bad boundary");
    if (p->boundary == DRTS_FRESNEL && !(p->n_outside > 0.0)) return fail(nullptr, DRTS_EINVAL, "n_outside must be > 0");
    if (p->precision < DRTS_FP64 || p->precision > DRTS_FP16_ROWSCALE) return fail(nullptr, DRTS_EINVAL, "bad precision");
    if (p->n_rhs < 1 || p->n_rhs > kMaxRhs) return fail(nullptr, DRTS_EINVAL, "n_rhs must be 1..64");
    if (p->det_face != DRTS_FACE_NONE) {
        if (p->det_face < 0 || p->det_face > 5) return fail(nullptr, DRTS_EINVAL, "bad det_face");
        const int N[3] = {p->nx, p->ny, p->nz};
        const int fa = p->det_face / 2, ua = fa == 0 ? 1 : 0, va = fa == 2 ? 1 : 2;
        if (p->det_nu < 1 || p->det_nv < 1 || p->det_nu > N[ua] || p->det_nv > N[va])
            return fail(nullptr, DRTS_EINVAL, "detector patch grid must be 1..side");
    }
    if (p->max_steps < 0) return fail(nullptr, DRTS_EINVAL, "max_steps < 0");
    if (p->batched_kernel != DRTS_BATCHED_CUDA_CORES && p->batched_kernel != DRTS_BATCHED_TENSOR)
        return fail(nullptr, DRTS_EINVAL, "bad batched_kernel");
    if (p->batched_kernel == DRTS_BATCHED_TENSOR && p->n_rhs > 1 && p->precision != DRTS_FP32)
        return fail(nullptr, DRTS_EUNSUPPORTED, "the tensor-core batched step runs FP32 problems");
    if (p->interface != DRTS_INTERFACE_FIRST_ORDER && p->interface != DRTS_INTERFACE_TWO_STEP)
        return fail(nullptr, DRTS_EINVAL, "bad interface");
    if (p->direction_weights != DRTS_HG_EQUAL && p->direction_weights != DRTS_HG_QUADRATURE)
        return fail(nullptr, DRTS_EINVAL, "bad direction_weights");
    if (p->interface == DRTS_INTERFACE_TWO_STEP) {
        // planar interfaces normal to z: one medium per z layer
        const int64_t layer = int64_t(p->nx) * p->ny;
        for (int64_t v = 0; v < V; ++v)
            if (p->medium_of_voxel[v] != p->medium_of_voxel[v - v % layer])
                return fail(nullptr, DRTS_EINVAL, "two-step interfaces need one medium per z layer");
    }
    return DRTS_OK;
}

drts_status sync_check(drts_ctx *c, const char *where)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    if (c->d_err) {
        int err = 0;
        e = cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, where);
        if (err) {
            cudaMemset(c->d_err, 0, sizeof(int));
            return fail(c, DRTS_ETIMEOUT, std::string(where) + ": a bounded device-side wait gave up");
        }
    }
    return DRTS_OK;
}

drts_status upload_sources(drts_ctx *c)
{
    // flatten profiles
    std::vector<double> vals;
    for (int r = 0; r < c->R; ++r) {
        c->prof[r].off = int32_t(vals.size());
        vals.insert(vals.end(), c->prof_vals[r].begin(), c->prof_vals[r].end());
    }
    std::sort(c->src.begin(), c->src.end(), [](const SourceEntry &a, const SourceEntry &b) {
        if (a.slice != b.slice) return a.slice < b.slice;
        if (a.lane != b.lane) return a.lane < b.lane;
        return a.rhs < b.rhs;
    });
    cudaError_t e = cudaSuccess;
    if (int64_t(vals.size()) > c->prof_cap) {
        int64_t cap = int64_t(vals.size()) * 2 + 16;
        double *p = nullptr;
        e = dalloc(c, &p, size_t(cap) * sizeof(double));
        if (e != cudaSuccess) return cuda_fail(c, e, "profile allocation");
        c->d_prof_vals = p;
        c->prof_cap = cap;
    }
    if (!vals.empty())
        e = cudaMemcpyAsync(c->d_prof_vals, vals.data(), vals.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !c->src.empty())
        e = cudaMemcpyAsync(c->d_src, c->src.data(), c->src.size() * sizeof(SourceEntry), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && c->d_src_voxel) {
        e = cudaMemsetAsync(c->d_src_voxel, 0, size_t(c->V), c->stream);
        std::vector<int64_t> vox;
        for (const SourceEntry &se : c->src) vox.push_back((int64_t(se.slice) / kDirs) * kSlice + se.lane);
        std::sort(vox.begin(), vox.end());
        vox.erase(std::unique(vox.begin(), vox.end()), vox.end());
        for (size_t q = 0; q < vox.size() && e == cudaSuccess; ++q)
            e = cudaMemsetAsync(c->d_src_voxel + vox[q], 1, 1, c->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_prof, c->prof.data(), c->prof.size() * sizeof(SourceProfile), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "source upload");
    return sync_check(c, "source upload");
}

// Right-hand side r inside a state buffer: first element and the distance
// between consecutive states (1 for one right-hand side; 4 for the batched
// layout, which keeps groups of four right-hand sides side by side).
struct RhsView {
    void *base;
    int stride;
};
RhsView rhs_view(drts_ctx *c, void *buf, int r)
{
    if (c->R == 1) return RhsView{buf, 1};
    const size_t elems = (size_t(r >> 2) * c->rhs_stride) * 4 + size_t(r & 3);
    return RhsView{static_cast<char *>(buf) + elems * state_elem_bytes(c->prob.precision), 4};
}

StepArgs make_args(drts_ctx *c)
{
    StepArgs a{};
    a.A = c->A;
    a.nx = c->prob.nx; a.ny = c->prob.ny; a.nz = c->prob.nz;
    a.V = c->V;
    a.R = c->R;
    a.rhs_stride = c->rhs_stride;
    a.tcp = c->tcp;
    a.src_voxel = c->d_src_voxel;
    a.x = c->x; a.y = c->y;
    a.cls = c->d_cls;
    a.tab.absorb = c->d_absorb;
    a.tab.absorb_dir = c->d_absorb_dir;
    a.tab.exit_total = c->d_exit_tot;
    a.tab.exit_det = c->d_exit_det;
    a.det_face = c->prob.det_face;
    a.det_nu = c->prob.det_nu; a.det_nv = c->prob.det_nv;
    a.n_patch = c->n_patch;
    a.det = nullptr;
    if (c->det && c->n_patch > 0 && c->t < c->prob.max_steps) a.det = c->det + c->t * c->n_patch;
    a.det_stride_r = c->prob.max_steps * c->n_patch;
    a.t = c->t;
    a.ledger = c->ledger;
    a.n_src = int(c->src.size());
    a.src = c->d_src;
    a.prof = c->d_prof;
    a.prof_vals = c->d_prof_vals;
    a.rhs_tile = c->rhs_tile;
    a.err = c->d_err;
    a.spin_limit = c->spin_limit;
    a.fault_skip_chunk = c->fault_skip_chunk;
    a.tcx = c->tc ? 1 : 0;
    a.pd.n_det = c->n_pdet;
    a.pd.off = c->d_pdet_off;
    a.pd.state = c->d_pdet_state;
    a.pd.w = c->d_pdet_w;
    a.pd.hist = (c->n_pdet > 0 && c->t < c->prob.max_steps) ? c->d_pdet_hist : nullptr;
    a.pd.stride_r = c->prob.max_steps * c->n_pdet;
    a.bulk.n_groups = c->n_bulk_groups;
    a.bulk.groups = c->d_bulk_groups;
    a.bulk.rhs_off = c->d_bulk_rhs_off;
    a.bulk.entries = c->d_bulk_entries;
    a.bulk.prof = c->d_bulk_prof;
    a.bulk.prof_vals = c->d_bulk_prof_vals;
    return a;
}

// One step from x(t): point detectors of x(t), the product with the fused
// source / face-detector / ledger terms, then the sub-step sources.
cudaError_t launch_any_step(drts_ctx *c, const StepArgs &a)
{
    cudaError_t e = launch_point_detectors(a, c->stream);
    if (e != cudaSuccess) return e;
    if (c->R == 1) e = launch_step(a, c->variant, c->blocks, c->threads, c->stream);
    else if (c->tc) e = launch_tc_step(a, true, c->stream);
    else e = launch_batched_step(a, c->R, c->rhs_tile, c->variant, c->blocks, c->threads, true, c->stream);
    if (e != cudaSuccess) return e;
    return launch_bulk_sources(a, c->stream);
}

int fit_blocks(drts_ctx *c, int threads, int variant, int rhs_tile)
{
    if (c->R == 1 && (variant == 7 || variant == 8) && c->prob.nx % kSlice != 0) return 0;   // halo: whole blocks
    if (c->R == 1) return step_default_blocks(c->A.precision, c->R, threads, variant);
    int dev = 0, sms = 0;
    if (c->tc) {
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return sms * tc_blocks_per_sm(nullptr);
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * batched_blocks_per_sm(c->A.precision, rhs_tile, threads, variant);
}

}  // namespace

namespace drts {
// The serving loop borrows a context's stream while capturing its steps.
cudaStream_t ctx_swap_stream(drts_ctx *c, cudaStream_t s)
{
    cudaStream_t old = c->stream;
    c->stream = s;
    return old;
}
}  // namespace drts

namespace {

// Tensor-core batched step: the union of each block role's (n, m) positions
// over all voxels (from the assembled sliced matrix), and A stored per voxel
// and role at those positions as three bf16 terms (drts_tensor.cu).
drts_status setup_tensor_core(drts_ctx *c)
{
    constexpr int kFlags = kOffs * kDirs * kDirs;
    uint8_t *dflags = nullptr;
    cudaError_t e = dalloc(c, &dflags, kFlags);
    if (e == cudaSuccess) e = cudaMemsetAsync(dflags, 0, kFlags, c->stream);
    if (e == cudaSuccess) e = launch_tc_flags(c->A, c->V, dflags, c->stream);
    std::vector<uint8_t> flags(kFlags, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flags.data(), dflags, kFlags, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core union pattern");
    drelease(c, dflags);
    // positions of each role in (m, n) order, padded to a multiple of 8 (16-byte
    // arrays); a role's chunk is three bf16 arrays
    std::vector<uint16_t> pos;
    std::vector<int16_t> pidx(kFlags, -1);
    TcPlan &P = c->tcp;
    int64_t off = 0;
    for (int d = 0; d < kOffs; ++d) {
        P.role_off[d] = int(pos.size());
        P.chunk_off[d] = int(off);
        int np = 0;
        for (int m = 0; m < kDirs; ++m)
            for (int n = 0; n < kDirs; ++n)
                if (flags[size_t(d) * kDirs * kDirs + n * kDirs + m]) {
                    pidx[size_t(d) * kDirs * kDirs + n * kDirs + m] = int16_t(np++);
                    pos.push_back(uint16_t((n << 8) | m));
                }
        while (np % 8) {
            pos.push_back(uint16_t(31 << 8));         // padding: direction slot 31 of the tile is zero
            ++np;
        }
        off += 6 * int64_t(np);
    }
    P.role_off[kOffs] = int(pos.size());
    P.chunk_off[kOffs] = int(off);
    P.voxel_bytes = off;
    if (P.role_off[kOffs] > tc_position_limit())
        return fail(c, DRTS_EUNSUPPORTED, "tensor-core step: the matrix's block pattern has more positions than "
                                          "the kernel's table holds");
    for (int L = 0; L < kOffs / 3; ++L)
        if (P.chunk_off[3 * L + 3] - P.chunk_off[3 * L] > tc_stage_limit())
            return fail(c, DRTS_EUNSUPPORTED, "tensor-core step: the matrix's block pattern needs more staging "
                                              "than one tile slot holds");
    uint16_t *dpos = nullptr;
    int16_t *dpidx = nullptr;
    void *dAu = nullptr;
    const size_t au_bytes = size_t(c->V) * size_t(P.voxel_bytes);
    if ((e = upload(c, &dpos, pos)) != cudaSuccess || (e = upload(c, &dpidx, pidx)) != cudaSuccess ||
        (e = dalloc(c, &dAu, au_bytes)) != cudaSuccess)
        return cuda_fail(c, e, "tensor-core matrix allocation");
    P.pos = dpos;
    P.Au = dAu;
    if ((e = cudaMemsetAsync(dAu, 0, au_bytes, c->stream)) != cudaSuccess ||
        (e = launch_tc_convert(c->A, c->V, dpidx, P, dAu, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "tensor-core matrix conversion");
    drelease(c, dpidx);
    std::string why;
    if (tc_blocks_per_sm(&why) < 1) return fail(c, DRTS_ECUDA, "tensor-core step kernel does not fit on an SM (" + why + ")");
    return DRTS_OK;
}

}  // namespace

void drts::set_global_error(const std::string &msg)
{
    g_assemble_error = msg;
}

extern "C" {

drts_status drts_assemble(const drts_problem *prob, void *cuda_stream, drts_ctx **out)
try {
    NvtxRange nvtx("drts_assemble");
    if (!out) return fail(nullptr, DRTS_EINVAL, "out is NULL");
    *out = nullptr;
    drts_status st = validate(prob);
    if (st != DRTS_OK) return st;
    drts_ctx *c = new (std::nothrow) drts_ctx;
    if (!c) return fail(nullptr, DRTS_ENOMEM, "host allocation");
    c->prob = *prob;
    c->prob.media = nullptr;
    c->prob.medium_of_voxel = nullptr;
    c->media.assign(prob->media, prob->media + prob->n_media);
    c->substep.assign(size_t(prob->n_rhs), drts_ctx::SubstepSource());
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->V = int64_t(prob->nx) * prob->ny * prob->nz;
    c->n_states = c->V * kDirs;
    c->K = prob->n_media;
    c->R = prob->n_rhs;
    c->rhs_stride = c->n_states + 64;     // the tail keeps padding lanes in bounds
    c->tc = prob->n_rhs > 1 && prob->batched_kernel == DRTS_BATCHED_TENSOR;
    if (prob->det_face != DRTS_FACE_NONE) c->n_patch = prob->det_nu * prob->det_nv;

    // a host allocation that throws below must not leak the partial context
    struct Unwind {
        drts_ctx *c;
        ~Unwind() { if (c) drts_destroy(c); }
    } unwind{c};
    auto bail = [&](drts_status s) {
        g_assemble_error = c->err;
        unwind.c = nullptr;
        drts_destroy(c);
        return s;
    };

    std::string terr = build_host_tables(*prob, c->host);
    if (!terr.empty()) {
        fail(c, DRTS_EINVAL, terr);
        return bail(DRTS_EINVAL);
    }
    const HostTables &H = c->host;
    cudaError_t e;
    // tables
    std::vector<uint8_t> med(prob->medium_of_voxel, prob->medium_of_voxel + c->V);
    double *dW, *dtv, *dre, *dri, *dnr;
    int32_t *dto;
    uint8_t *dtn, *dmed, *dplain;
    if ((e = upload(c, &dW, H.W)) != cudaSuccess ||
        (e = upload(c, &dto, H.tmpl_off)) != cudaSuccess ||
        (e = upload(c, &dtn, H.tmpl_n)) != cudaSuccess ||
        (e = upload(c, &dtv, H.tmpl_val)) != cudaSuccess ||
        (e = upload(c, &dre, H.r_edge)) != cudaSuccess ||
        (e = upload(c, &dri, H.r_int)) != cudaSuccess ||
        (e = upload(c, &dnr, H.nref)) != cudaSuccess ||
        (e = upload(c, &dmed, med)) != cudaSuccess ||
        (e = dalloc(c, &dplain, size_t(c->V))) != cudaSuccess ||
        (e = upload(c, &c->d_absorb, H.led_absorb)) != cudaSuccess ||
        (e = upload(c, &c->d_exit_tot, H.led_exit_total)) != cudaSuccess ||
        (e = upload(c, &c->d_exit_det, H.led_exit_det)) != cudaSuccess) {
        cuda_fail(c, e, "table upload");
        return bail(e == cudaErrorMemoryAllocation ? DRTS_ENOMEM : DRTS_ECUDA);
    }
    DevTables &T = c->T;
    T.nx = prob->nx; T.ny = prob->ny; T.nz = prob->nz;
    T.V = c->V; T.K = c->K;
    T.W = dW; T.tmpl_off = dto; T.tmpl_n = dtn; T.tmpl_val = dtv;
    T.r_edge = dre; T.r_int = dri; T.nref = dnr; T.med = dmed; T.plain = dplain;
    c->d_med = dmed;
    c->d_cls = dmed;
    c->med_host = med;
    if (prob->interface == DRTS_INTERFACE_TWO_STEP) {
        // pair tables for the assembler, per-layer ledger classes for the step
        const int64_t layer = int64_t(prob->nx) * prob->ny;
        c->cls_host.resize(size_t(c->V));
        for (int64_t v = 0; v < c->V; ++v) c->cls_host[size_t(v)] = H.class_of_layer[size_t(v / layer)];
        int32_t *dps = nullptr;
        uint8_t *dcr = nullptr;
        double *dw2f = nullptr, *dw2n = nullptr;
        if ((e = upload(c, &dps, H.pair_slot)) != cudaSuccess ||
            (H.n_pairs > 0 && ((e = upload(c, &dcr, H.cross)) != cudaSuccess ||
                               (e = upload(c, &dw2f, H.W2f)) != cudaSuccess ||
                               (e = upload(c, &dw2n, H.W2n)) != cudaSuccess)) ||
            (e = upload(c, &c->d_absorb_dir, H.led_absorb_dir)) != cudaSuccess ||
            (e = upload(c, &c->d_cls, c->cls_host)) != cudaSuccess) {
            cuda_fail(c, e, "two-step table upload");
            return bail(e == cudaErrorMemoryAllocation ? DRTS_ENOMEM : DRTS_ECUDA);
        }
        T.interface = DRTS_INTERFACE_TWO_STEP;
        T.pair_slot = dps; T.cross = dcr; T.W2f = dw2f; T.W2n = dw2n;
    }

    // slices and counts
    SlicedMatrix &A = c->A;
    A.precision = prob->precision;
    A.n_slices = ((c->V + kSlice - 1) / kSlice) * kDirs;
    int64_t *d_total = nullptr;
    unsigned long long *d_split = nullptr;
    if ((e = dalloc(c, &A.slice_ptr, sizeof(int64_t) * A.n_slices)) != cudaSuccess ||
        (e = dalloc(c, &A.slice_len4, sizeof(int32_t) * A.n_slices)) != cudaSuccess ||
        (e = dalloc(c, &A.row_len, sizeof(int32_t) * A.n_slices * kSlice)) != cudaSuccess ||
        (e = dalloc(c, &d_total, sizeof(int64_t))) != cudaSuccess ||
        (e = dalloc(c, &d_split, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMemsetAsync(d_split, 0, sizeof(unsigned long long), c->stream)) != cudaSuccess) {
        cuda_fail(c, e, "slice table allocation");
        return bail(DRTS_ENOMEM);
    }
    if (prob->precision == DRTS_FP16_ROWSCALE) {
        float *dscale = nullptr;
        if ((e = upload(c, &dscale, H.dir_scale)) != cudaSuccess ||
            (e = dalloc(c, &A.row_scale, sizeof(float) * A.n_slices * kSlice)) != cudaSuccess) {
            cuda_fail(c, e, "row scale allocation");
            return bail(DRTS_ENOMEM);
        }
        T.dir_scale = dscale;
    }
    if ((e = launch_classify(T, dplain, c->stream)) != cudaSuccess ||
        (e = launch_count(T, A, d_split, c->stream)) != cudaSuccess ||
        (e = launch_scan(A, d_total, c->stream)) != cudaSuccess) {
        cuda_fail(c, e, "assembly count");
        return bail(DRTS_ECUDA);
    }
    int64_t groups = 0;
    unsigned long long n_split = 0;
    if ((e = cudaMemcpyAsync(&groups, d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&n_split, d_split, sizeof(n_split), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
        cuda_fail(c, e, "assembly count");
        return bail(DRTS_ECUDA);
    }
    A.n_groups = groups;
    const size_t slots = size_t(groups) * kSlice * kGroup;
    if ((e = dalloc(c, &A.vals, slots * value_bytes(A.precision))) != cudaSuccess ||
        (e = dalloc(c, &A.codes, slots * sizeof(uint16_t))) != cudaSuccess) {
        cuda_fail(c, e, ("matrix allocation (" + std::to_string(slots) + " slots)").c_str());
        return bail(DRTS_ENOMEM);
    }
    if ((e = launch_fill(T, A, c->stream)) != cudaSuccess) {
        cuda_fail(c, e, "assembly fill");
        return bail(DRTS_ECUDA);
    }
    // nnz and special-voxel share (host reductions of small device arrays)
    {
        std::vector<int32_t> rl(size_t(A.n_slices) * kSlice);
        std::vector<uint8_t> pl(size_t(c->V));
        if ((e = cudaMemcpyAsync(rl.data(), A.row_len, rl.size() * 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(pl.data(), dplain, pl.size(), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
            cuda_fail(c, e, "assembly readback");
            return bail(DRTS_ECUDA);
        }
        int64_t nnz = 0, special = 0;
        for (int32_t x : rl) nnz += x;
        for (uint8_t x : pl) special += x == 0;
        A.nnz = nnz;
        A.nnz_stored = nnz + int64_t(n_split);
        c->special_permille = int(special * 1000 / c->V);
    }
    // state, ledger, detector history, sources
    c->x_elems = c->tc ? int64_t(tcx_state_bytes(c->V) / 4)
                       : (c->R == 1 ? c->rhs_stride : c->rhs_stride * ((c->R + 3) / 4) * 4);
    if (c->tc) {
        st = setup_tensor_core(c);
        if (st != DRTS_OK) return bail(st);
    }
    const size_t sb = size_t(c->x_elems) * state_elem_bytes(prob->precision);
    if ((e = dalloc(c, &c->x, sb)) != cudaSuccess || (e = dalloc(c, &c->y, sb)) != cudaSuccess ||
        (e = dalloc(c, &c->ledger, sizeof(double) * 4 * c->R)) != cudaSuccess ||
        (e = dalloc(c, &c->d_src, sizeof(SourceEntry) * kMaxSrc * c->R)) != cudaSuccess ||
        (e = dalloc(c, &c->d_prof, sizeof(SourceProfile) * c->R)) != cudaSuccess ||
        (e = dalloc(c, &c->d_err, sizeof(int))) != cudaSuccess ||
        (e = dalloc(c, &c->d_bar, 2 * sizeof(unsigned))) != cudaSuccess ||
        (e = dalloc(c, &c->d_src_voxel, size_t(c->V))) != cudaSuccess) {
        cuda_fail(c, e, "state allocation");
        return bail(DRTS_ENOMEM);
    }
    if (c->n_patch > 0 && prob->max_steps > 0) {
        if ((e = dalloc(c, &c->det, sizeof(double) * size_t(c->R) * prob->max_steps * c->n_patch)) != cudaSuccess) {
            cuda_fail(c, e, "detector allocation");
            return bail(DRTS_ENOMEM);
        }
        cudaMemsetAsync(c->det, 0, sizeof(double) * size_t(c->R) * prob->max_steps * c->n_patch, c->stream);
    }
    cudaMemsetAsync(c->x, 0, sb, c->stream);
    cudaMemsetAsync(c->y, 0, sb, c->stream);
    cudaMemsetAsync(c->ledger, 0, sizeof(double) * 4 * c->R, c->stream);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    cudaMemsetAsync(c->d_src_voxel, 0, size_t(c->V), c->stream);
    c->prof.assign(c->R, SourceProfile{0, 0, 0, 0, 0});
    c->prof_vals.assign(c->R, std::vector<double>());
    st = upload_sources(c);
    if (st != DRTS_OK) return bail(st);
    c->threads = 256;
    c->variant = 0;
    c->rhs_tile = 0;
    if (c->R > 1 && !c->tc) {
        // measured default of the CUDA-core batched step (GB300, FP32, grids
        // 48^3 - 96^3): 8 right-hand sides per pass (two 16-byte gathers per
        // nonzero), warps striding over the slices (the autotuner refines
        // this per problem)
        c->rhs_tile = c->R <= 4 ? 4 : 8;
    }
    if (c->tc) c->rhs_tile = kMaxRhs;      // all right-hand sides in one pass
    c->blocks = fit_blocks(c, c->threads, c->variant, c->rhs_tile);
    if (c->blocks < 1) {
        fail(c, DRTS_ECUDA, "step kernel does not fit on an SM");
        return bail(DRTS_ECUDA);
    }
    st = sync_check(c, "assembly");
    if (st != DRTS_OK) return bail(st);
    unwind.c = nullptr;
    *out = c;
    return DRTS_OK;
} catch (...) {
    return caught(nullptr, "drts_assemble");
}

drts_status drts_inject_source(drts_ctx *c, int32_t rhs, int32_t n_entries, const int64_t *state_idx,
                               const double *weight, int64_t t0, int32_t n_t, const double *profile)
try {
    if (!c) return DRTS_EINVAL;
    if (rhs < 0 || rhs >= c->R) return fail(c, DRTS_EINVAL, "rhs out of range");
    if (n_entries < 0 || n_entries > kMaxSrc) return fail(c, DRTS_EINVAL, "n_entries must be 0..64");
    if (n_t < 0 || (n_t > 0 && !profile)) return fail(c, DRTS_EINVAL, "bad profile");
    if (n_entries > 0 && (!state_idx || !weight)) return fail(c, DRTS_EINVAL, "NULL source arrays");
    std::vector<SourceEntry> keep;
    for (const SourceEntry &e : c->src)
        if (e.rhs != rhs) keep.push_back(e);
    for (int i = 0; i < n_entries; ++i) {
        const int64_t s = state_idx[i];
        if (s < 0 || s >= c->n_states) return fail(c, DRTS_EINVAL, "source state out of range");
        if (!std::isfinite(weight[i])) return fail(c, DRTS_EINVAL, "source weight not finite");
        const int64_t v = s / kDirs;
        const int d = int(s % kDirs);
        SourceEntry e{};
        e.slice = int32_t((v / kSlice) * kDirs + d);
        e.lane = int32_t(v % kSlice);
        e.rhs = rhs;
        e.prof = rhs;
        e.w = weight[i];
        keep.push_back(e);
    }
    if (int(keep.size()) > kMaxSrc * c->R) return fail(c, DRTS_EINVAL, "too many source entries");
    c->src = keep;
    c->prof[rhs] = SourceProfile{t0, n_t, 0, 0, 0};
    c->prof_vals[rhs].assign(profile, profile + n_t);
    return upload_sources(c);
} catch (...) {
    return caught(c, "drts_inject_source");
}

drts_status drts_step_n(drts_ctx *c, int64_t n_steps)
try {
    NvtxRange nvtx("drts_step_n");
    if (!c) return DRTS_EINVAL;
    if (n_steps < 0) return fail(c, DRTS_EINVAL, "n_steps < 0");
    if ((c->det || c->n_pdet > 0) && c->t + n_steps > c->prob.max_steps)
        return fail(c, DRTS_EINVAL, "t + n_steps exceeds max_steps");
    if (c->step_mode == DRTS_STEP_PERSISTENT && n_steps > 0) {
        if (c->n_bulk_groups > 0)
            return fail(c, DRTS_EUNSUPPORTED, "sub-step sources need the launch step mode");
        StepArgs a = make_args(c);
        // the launch path's split variants (two or four warps per slice) carry over
        int split = c->variant == 10 ? 2 : (c->variant == 11 ? 4 : (c->variant == 14 ? 8 : 1));
        if (c->threads / 32 < split) split = 1;
        // as many blocks as the launch path uses, when they can all be resident
        int blocks = persistent_blocks(c->prob.precision, c->threads, split);
        if (blocks < 1) return fail(c, DRTS_EUNSUPPORTED, "persistent kernel does not fit");
        if (c->blocks > 0 && c->blocks < blocks) blocks = c->blocks;
        cudaError_t e = launch_persistent(a, c->y, n_steps, c->det, c->prob.max_steps, c->d_bar,
                                          c->fault_skip_barrier, blocks, c->threads, split, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "persistent launch");
        if (n_steps & 1) std::swap(c->x, c->y);
        c->t += n_steps;
        return DRTS_OK;
    }
    for (int64_t i = 0; i < n_steps; ++i) {
        StepArgs a = make_args(c);
        cudaError_t e = launch_any_step(c, a);
        if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
        std::swap(c->x, c->y);
        ++c->t;
    }
    return DRTS_OK;
} catch (...) {
    return caught(c, "drts_step_n");
}

drts_status drts_run_host(drts_ctx *c, int64_t n_steps, const double *scale, double *det_out)
try {
    NvtxRange nvtx("drts_run_host");
    if (!c) return DRTS_EINVAL;
    if (n_steps < 0 || !scale) return fail(c, DRTS_EINVAL, "bad arguments");
    if (c->n_bulk_groups > 0)
        return fail(c, DRTS_EUNSUPPORTED, "run_host scales the plain sources; sub-step sources are set");
    if ((c->det || c->n_pdet > 0) && c->t + n_steps > c->prob.max_steps)
        return fail(c, DRTS_EINVAL, "t + n_steps exceeds max_steps");
    if (n_steps == 0) return DRTS_OK;
    double *d_scale = nullptr;
    cudaError_t e = cudaMallocAsync(&d_scale, sizeof(double) * c->R * n_steps, c->stream);
    for (int64_t i = 0; i < n_steps && e == cudaSuccess; ++i) {
        // this step's source factors, host -> device
        e = cudaMemcpyAsync(d_scale + i * c->R, scale + i * c->R, sizeof(double) * c->R,
                            cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) break;
        StepArgs a = make_args(c);
        a.step_scale = d_scale + i * c->R;
        e = launch_any_step(c, a);
        if (e != cudaSuccess) break;
        // this step's detector readout, device -> host
        if (det_out && a.det && c->n_patch > 0)
            for (int r = 0; r < c->R && e == cudaSuccess; ++r)
                e = cudaMemcpyAsync(det_out + (i * c->R + r) * c->n_patch, a.det + r * a.det_stride_r,
                                    sizeof(double) * c->n_patch, cudaMemcpyDeviceToHost, c->stream);
        std::swap(c->x, c->y);
        ++c->t;
    }
    if (d_scale) cudaFreeAsync(d_scale, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "run_host");
    return sync_check(c, "run_host");
} catch (...) {
    return caught(c, "drts_run_host");
}

drts_status drts_read_detectors(drts_ctx *c, int32_t rhs, int64_t t_begin, int64_t t_end, double *host_out,
                                double *ledger_out)
try {
    if (!c) return DRTS_EINVAL;
    if (rhs < 0 || rhs >= c->R) return fail(c, DRTS_EINVAL, "rhs out of range");
    if (t_begin < 0 || t_end < t_begin || t_end > c->t) return fail(c, DRTS_EINVAL, "bad step range");
    cudaError_t e = cudaSuccess;
    if (t_end > t_begin) {
        if (!c->det) return fail(c, DRTS_ESTATE, "no detector history (det_face none or max_steps 0)");
        if (!host_out) return fail(c, DRTS_EINVAL, "host_out is NULL");
        e = cudaMemcpyAsync(host_out, c->det + (size_t(rhs) * c->prob.max_steps + t_begin) * c->n_patch,
                            sizeof(double) * (t_end - t_begin) * c->n_patch, cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess && ledger_out) {
        double *tmp = nullptr;
        e = cudaMallocAsync(&tmp, sizeof(double), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(tmp, 0, sizeof(double), c->stream);
        if (e == cudaSuccess) e = (c->tc ? launch_tc_sum(c->x, c->V, rhs, tmp, c->stream)
                                      : launch_ledger_sum(rhs_view(c, c->x, rhs).base, c->prob.precision, c->n_states,
                                                          rhs_view(c, c->x, rhs).stride, 0, tmp, c->stream));
        if (e == cudaSuccess) e = cudaMemcpyAsync(ledger_out, tmp, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ledger_out + 1, c->ledger + 4 * rhs + 1, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (tmp) cudaFreeAsync(tmp, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "read_detectors");
    return sync_check(c, "read_detectors");
} catch (...) {
    return caught(c, "drts_read_detectors");
}

drts_status drts_read_state(drts_ctx *c, int32_t rhs, double *host_out)
try {
    if (!c) return DRTS_EINVAL;
    if (rhs < 0 || rhs >= c->R || !host_out) return fail(c, DRTS_EINVAL, "bad arguments");
    double *tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, sizeof(double) * c->n_states, c->stream);
    if (e == cudaSuccess)
        e = c->tc ? launch_tc_to_canonical(c->x, c->V, rhs, tmp, c->stream)
                  : launch_to_canonical(rhs_view(c, c->x, rhs).base, c->prob.precision, c->V,
                                        rhs_view(c, c->x, rhs).stride, 0, tmp, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, tmp, sizeof(double) * c->n_states, cudaMemcpyDeviceToHost, c->stream);
    if (tmp) cudaFreeAsync(tmp, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "read_state");
    return sync_check(c, "read_state");
} catch (...) {
    return caught(c, "drts_read_state");
}

drts_status drts_write_state(drts_ctx *c, int32_t rhs, const double *host_in)
try {
    if (!c) return DRTS_EINVAL;
    if (rhs < 0 || rhs >= c->R || !host_in) return fail(c, DRTS_EINVAL, "bad arguments");
    double *tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, sizeof(double) * c->n_states, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tmp, host_in, sizeof(double) * c->n_states, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = c->tc ? launch_tc_from_canonical(tmp, c->V, rhs, c->x, c->stream)
                  : launch_from_canonical(tmp, c->prob.precision, c->V, rhs_view(c, c->x, rhs).stride, 0,
                                          rhs_view(c, c->x, rhs).base, c->stream);
    if (tmp) cudaFreeAsync(tmp, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "write_state");
    return sync_check(c, "write_state");
} catch (...) {
    return caught(c, "drts_write_state");
}

drts_status drts_export_rows(drts_ctx *c, int64_t row_begin, int64_t row_end, int64_t *row_ptr, int32_t *col,
                             double *val, int64_t cap)
try {
    if (!c) return DRTS_EINVAL;
    if (row_begin < 0 || row_end < row_begin || row_end > c->n_states || !row_ptr)
        return fail(c, DRTS_EINVAL, "bad row range");
    const int64_t n = row_end - row_begin;
    std::vector<int64_t> cnt(size_t(n) + 1, 0);     // before the device buffer: a throw here leaks nothing
    int64_t *dcount = nullptr;
    cudaError_t e = cudaMallocAsync(&dcount, sizeof(int64_t) * (n + 1), c->stream);
    if (e == cudaSuccess) e = launch_count_export(c->A, c->V, row_begin, row_end, dcount, c->stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(cnt.data(), dcount, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        if (dcount) cudaFree(dcount);
        return cuda_fail(c, e, "export_rows");
    }
    row_ptr[0] = 0;
    for (int64_t r = 0; r < n; ++r) row_ptr[r + 1] = row_ptr[r] + cnt[size_t(r)];
    const int64_t nnz = row_ptr[n];
    if (nnz > cap || (nnz > 0 && (!col || !val))) {
        cudaFree(dcount);
        return fail(c, DRTS_EINVAL, "export capacity " + std::to_string(cap) + " < " + std::to_string(nnz));
    }
    int32_t *dcol = nullptr;
    double *dval = nullptr;
    e = cudaMemcpyAsync(dcount, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&dcol, sizeof(int32_t) * (nnz + 1), c->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&dval, sizeof(double) * (nnz + 1), c->stream);
    if (e == cudaSuccess)
        e = launch_export(c->A, c->prob.nx, c->prob.ny, c->prob.nz, row_begin, row_end, dcount, dcol, dval, c->stream);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(col, dcol, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(val, dval, sizeof(double) * nnz, cudaMemcpyDeviceToHost, c->stream);
    if (dcol) cudaFreeAsync(dcol, c->stream);
    if (dval) cudaFreeAsync(dval, c->stream);
    cudaFreeAsync(dcount, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "export_rows");
    return sync_check(c, "export_rows");
} catch (...) {
    return caught(c, "drts_export_rows");
}

drts_status drts_host_tables(const drts_problem *prob, int32_t medium, double *stencil_out,
                             double *exit_total_out, double *exit_det_out, float *dir_scale_out)
try {
    drts_status st = validate(prob);
    if (st != DRTS_OK) return st;
    if (medium < 0 || medium >= prob->n_media) return fail(nullptr, DRTS_EINVAL, "medium out of range");
    HostTables H;
    const std::string err = build_host_tables(*prob, H);
    if (!err.empty()) return fail(nullptr, DRTS_EINVAL, err);
    const size_t nw = size_t(kDirs) * kOffs * kDirs, ne = size_t(27) * kDirs;
    if (stencil_out) std::memcpy(stencil_out, H.W.data() + size_t(medium) * nw, nw * sizeof(double));
    if (exit_total_out) std::memcpy(exit_total_out, H.exit_total.data() + size_t(medium) * ne, ne * sizeof(double));
    if (exit_det_out) std::memcpy(exit_det_out, H.exit_det.data() + size_t(medium) * ne, ne * sizeof(double));
    if (dir_scale_out) std::memcpy(dir_scale_out, H.dir_scale.data(), kDirs * sizeof(float));
    return DRTS_OK;
} catch (...) {
    return caught(nullptr, "drts_host_tables");
}

drts_status drts_two_step_tables(const drts_problem *prob, int32_t k1, int32_t k2, uint8_t *cross_out,
                                 double *fold_out, double *edge_out)
try {
    drts_status st = validate(prob);
    if (st != DRTS_OK) return st;
    if (prob->interface != DRTS_INTERFACE_TWO_STEP)
        return fail(nullptr, DRTS_EINVAL, "interface is not DRTS_INTERFACE_TWO_STEP");
    if (k1 < 0 || k1 >= prob->n_media || k2 < 0 || k2 >= prob->n_media)
        return fail(nullptr, DRTS_EINVAL, "medium out of range");
    HostTables H;
    const std::string err = build_host_tables(*prob, H);
    if (!err.empty()) return fail(nullptr, DRTS_EINVAL, err);
    const int q = H.pair_slot[size_t(k1) * prob->n_media + k2];
    if (q < 0) return fail(nullptr, DRTS_EINVAL, "the media do not meet across a z plane with different indices");
    const size_t nw = size_t(kDirs) * kOffs * kDirs;
    if (cross_out) std::memcpy(cross_out, H.cross.data() + size_t(q) * kDirs, kDirs);
    if (fold_out) std::memcpy(fold_out, H.W2f.data() + size_t(q) * nw, nw * sizeof(double));
    if (edge_out) std::memcpy(edge_out, H.W2n.data() + size_t(q) * nw, nw * sizeof(double));
    return DRTS_OK;
} catch (...) {
    return caught(nullptr, "drts_two_step_tables");
}

drts_status drts_column_info(drts_ctx *c, double *absorb, double *exit_total, double *exit_det)
try {
    if (!c) return DRTS_EINVAL;
    // host evaluation of the per-(ledger class, face mask, direction) tables
    // the step reads, over the class map on the device (a one-off readout,
    // not part of the step)
    std::vector<uint8_t> cls(size_t(c->V));
    cudaError_t e = cudaMemcpyAsync(cls.data(), c->d_cls, size_t(c->V), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "column_info");
    const HostTables &H = c->host;
    const int nx = c->prob.nx, ny = c->prob.ny, nz = c->prob.nz;
    for (int64_t v = 0; v < c->V; ++v) {
        const int x = int(v % nx), y = int(v / nx % ny), z = int(v / (int64_t(nx) * ny));
        const int b[3] = {x == 0 ? 0 : (x == nx - 1 ? 2 : 1), y == 0 ? 0 : (y == ny - 1 ? 2 : 1),
                          z == 0 ? 0 : (z == nz - 1 ? 2 : 1)};
        const int mask = b[2] * 9 + b[1] * 3 + b[0];
        const int k = cls[size_t(v)];
        for (int d = 0; d < kDirs; ++d) {
            const size_t ti = (size_t(k) * 27 + mask) * kDirs + d;
            if (absorb)
                absorb[v * kDirs + d] = H.led_absorb_dir.empty() ? H.led_absorb[k] : H.led_absorb_dir[k * kDirs + d];
            if (exit_total) exit_total[v * kDirs + d] = H.led_exit_total[ti];
            if (exit_det) exit_det[v * kDirs + d] = H.led_exit_det[ti];
        }
    }
    return DRTS_OK;
} catch (...) {
    return caught(c, "drts_column_info");
}

drts_status drts_get_info(const drts_ctx *c, drts_info *out)
{
    if (!c || !out) return DRTS_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->n_states = c->n_states;
    out->nnz = c->A.nnz;
    out->nnz_stored = c->A.nnz_stored;
    out->nnz_padded = c->A.n_groups * kSlice * kGroup;
    out->n_slices = c->A.n_slices;
    out->matrix_bytes = out->nnz_padded * int64_t(value_bytes(c->A.precision) + sizeof(uint16_t)) +
                        c->A.n_slices * int64_t(sizeof(int64_t) + sizeof(int32_t)) +
                        (c->A.row_scale ? c->A.n_slices * kSlice * 4 : 0);
    out->state_bytes = c->x_elems * int64_t(state_elem_bytes(c->A.precision));
    out->t = c->t;
    out->precision = c->A.precision;
    out->n_rhs = c->R;
    out->n_patch = c->n_patch;
    out->special_voxels_permille = c->special_permille;
    return DRTS_OK;
}

drts_status drts_set_launch(drts_ctx *c, int32_t blocks_per_sm, int32_t threads_per_block, int32_t rhs_tile,
                            int32_t variant)
try {
    if (!c) return DRTS_EINVAL;
    if (threads_per_block != 0 && (threads_per_block < 32 || threads_per_block > 256 || threads_per_block % 32))
        return fail(c, DRTS_EINVAL, "threads_per_block must be a multiple of 32 in 32..256");
    if (blocks_per_sm < 0 || blocks_per_sm > 64) return fail(c, DRTS_EINVAL, "blocks_per_sm must be 0..64");
    const int n_variants = c->R == 1 ? kStepVariants : (c->tc ? 1 : kBatchedOrders);
    if (variant < -1 || variant >= n_variants) return fail(c, DRTS_EINVAL, "unknown step variant");
    int tile = c->rhs_tile;
    if (c->R > 1 && rhs_tile != 0) {
        if (rhs_tile != 4 && rhs_tile != 8 && rhs_tile != 16 && rhs_tile != 32)
            return fail(c, DRTS_EINVAL, "rhs_tile must be 4, 8, 16 or 32");
        tile = c->tc ? c->rhs_tile : rhs_tile;     // the tensor-core form takes all rhs at once
    }
    const int threads = threads_per_block ? threads_per_block : 256;
    const int var = variant < 0 ? c->variant : variant;
    const int fit = fit_blocks(c, threads, var, tile);
    if (fit < 1) return fail(c, DRTS_EINVAL, "launch shape does not fit on an SM");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (blocks_per_sm && sms * blocks_per_sm > fit)
        return fail(c, DRTS_EINVAL, "more blocks per SM than fit (" + std::to_string(fit / sms) + ")");
    c->threads = threads;
    c->variant = var;
    c->rhs_tile = tile;
    c->blocks = blocks_per_sm ? sms * blocks_per_sm : fit;
    return DRTS_OK;
} catch (...) {
    return caught(c, "drts_set_launch");
}

namespace {

// Autotuner cache: (grid, precision, rhs, SM count, nnz) -> best launch.
std::mutex g_tune_mu;
std::map<std::string, drts_tune_result> g_tune_cache;

std::string tune_key(const drts_ctx *c, int sms)
{
    std::ostringstream k;
    k << c->prob.nx << 'x' << c->prob.ny << 'x' << c->prob.nz << ":p" << c->prob.precision << ":r" << c->R
      << ":sm" << sms << ":nnz" << c->A.nnz_stored;
    return k.str();
}

void tune_file_load(const char *path)
{
    std::ifstream f(path);
    std::string key;
    drts_tune_result r{};
    while (f >> key >> r.variant >> r.threads >> r.blocks_per_sm >> r.rhs_tile >> r.ms_per_step) {
        r.candidates = 0;
        r.from_cache = 1;
        g_tune_cache[key] = r;
    }
}

void tune_file_store(const char *path, const std::string &key, const drts_tune_result &r)
{
    std::ofstream f(path, std::ios::app);
    f << key << ' ' << r.variant << ' ' << r.threads << ' ' << r.blocks_per_sm << ' ' << r.rhs_tile << ' '
      << r.ms_per_step << '\n';
}

}  // namespace

drts_status drts_autotune(drts_ctx *c, int32_t trial_steps, drts_tune_result *out)
try {
    NvtxRange nvtx("drts_autotune");
    if (!c) return DRTS_EINVAL;
    if (trial_steps < 1 || trial_steps > 1000) return fail(c, DRTS_EINVAL, "trial_steps must be 1..1000");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const std::string key = tune_key(c, sms);
    const char *cache_path = std::getenv("DRTS_TUNE_CACHE");
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        if (cache_path && g_tune_cache.empty()) tune_file_load(cache_path);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            const drts_tune_result &r = it->second;
            drts_status st = drts_set_launch(c, r.blocks_per_sm, r.threads, r.rhs_tile, r.variant);
            if (st == DRTS_OK) {
                if (out) {
                    *out = r;
                    out->from_cache = 1;
                }
                return DRTS_OK;
            }
        }
    }
    // time every candidate on the current state without advancing it: the
    // step writes y from x (no swap), with no detector and a scratch ledger
    double *scratch_ledger = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&scratch_ledger, sizeof(double) * 4 * c->R);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    drts_tune_result best{};
    best.ms_per_step = 1e30;
    int tried = 0;
    // mean ms per step of one candidate over `steps` launches after one warm-up
    auto time_candidate = [&](const drts_tune_result &r, int steps, double &per) -> cudaError_t {
        StepArgs a = make_args(c);
        a.det = nullptr;
        a.ledger = scratch_ledger;
        a.n_src = 0;
        const int blocks = r.blocks_per_sm * sms;
        auto run = [&]() {
            if (c->R == 1) return launch_step(a, r.variant, blocks, r.threads, c->stream);
            if (c->tc) return launch_tc_step(a, false, c->stream);
            return launch_batched_step(a, c->R, r.rhs_tile > 0 ? r.rhs_tile : 4, r.variant, blocks, r.threads, false,
                                       c->stream);
        };
        cudaError_t err = run();          // warm-up
        if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
        for (int i = 0; i < steps && err == cudaSuccess; ++i) err = run();
        if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        per = double(ms) / steps;
        return err;
    };
    std::vector<drts_tune_result> cand;
    const int n_var = c->R == 1 ? kStepVariants : (c->tc ? 1 : kBatchedOrders);
    for (int var = 0; var < n_var && e == cudaSuccess; ++var)
        for (int tile : {4, 8, 16, 32})
        for (int threads : {256, 128}) {
            if (c->R == 1 && tile != 4) continue;             // tile only matters when batched
            if (c->tc && (tile != 4 || threads != 256)) continue;      // one fixed shape
            if (c->R > 1 && tile > 4 && tile / 2 >= c->R) continue;   // tile far wider than R
            if (c->R > 1 && !c->tc && var == 2 && (tile != 4 || threads != 256)) continue;   // fixed shape
            const int fit = fit_blocks(c, threads, var, tile);
            if (fit < 1) continue;
            const int fit_per_sm = fit / sms;
            for (int bps : {fit_per_sm, fit_per_sm / 2}) {
                if (bps < 1 || (bps == fit_per_sm / 2 && bps == fit_per_sm)) continue;
                drts_tune_result r{};
                r.variant = var;
                r.threads = threads;
                r.blocks_per_sm = bps;
                r.rhs_tile = c->R > 1 ? tile : 0;
                e = time_candidate(r, trial_steps, r.ms_per_step);
                if (e != cudaSuccess) break;
                ++tried;
                cand.push_back(r);
            }
        }
    // single short trials are noisy on a shared machine: the fastest few are
    // timed again, alternately, over three times the steps, and the best of
    // those repeats decides
    if (e == cudaSuccess && !cand.empty()) {
        std::stable_sort(cand.begin(), cand.end(),
                         [](const drts_tune_result &x, const drts_tune_result &y) { return x.ms_per_step < y.ms_per_step; });
        const size_t top = std::min<size_t>(cand.size(), 4);
        std::vector<double> rt(top, 1e30);
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep)
            for (size_t i = 0; i < top && e == cudaSuccess; ++i) {
                double per = 0.0;
                e = time_candidate(cand[i], 3 * trial_steps, per);
                rt[i] = std::min(rt[i], per);
            }
        for (size_t i = 0; i < top; ++i)
            if (rt[i] < best.ms_per_step) {
                best = cand[i];
                best.ms_per_step = rt[i];
            }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (scratch_ledger) cudaFree(scratch_ledger);
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
    drts_status st = sync_check(c, "autotune");
    if (st != DRTS_OK) return st;
    if (tried == 0) return fail(c, DRTS_ECUDA, "autotune: no candidate fits");
    best.candidates = tried;
    best.from_cache = 0;
    st = drts_set_launch(c, best.blocks_per_sm, best.threads, best.rhs_tile, best.variant);
    if (st != DRTS_OK) return st;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
        if (cache_path) tune_file_store(cache_path, key, best);
    }
    if (out) *out = best;
    return DRTS_OK;
} catch (...) {
    return caught(c, "drts_autotune");
}

namespace {
struct CheckpointHeader {
    uint64_t magic;                      // "DRTSCKP2"
    int32_t nx, ny, nz, precision, n_rhs, n_patch;
    int64_t nnz, t, max_steps;
    int32_t n_pdet, pad;
};
constexpr uint64_t kCkpMagic = 0x32504b4353545244ull;

int64_t checkpoint_bytes(const drts_ctx *c)
{
    return int64_t(sizeof(CheckpointHeader)) + int64_t(c->R) * (c->n_states * 8 + 4 * 8) +
           (c->det ? int64_t(c->R) * c->t * c->n_patch * 8 : 0) +
           (c->n_pdet > 0 ? int64_t(c->R) * c->t * c->n_pdet * 8 : 0);
}
}  // namespace

drts_status drts_checkpoint_size(drts_ctx *c, int64_t *bytes)
try {
    if (!c || !bytes) return DRTS_EINVAL;
    *bytes = checkpoint_bytes(c);
    return DRTS_OK;
} catch (...) {
    return caught(c, "drts_checkpoint_size");
}

drts_status drts_checkpoint_save(drts_ctx *c, void *host_buf, int64_t cap)
try {
    NvtxRange nvtx("drts_checkpoint_save");
    if (!c || !host_buf) return DRTS_EINVAL;
    const int64_t need = checkpoint_bytes(c);
    if (cap < need) return fail(c, DRTS_EINVAL, "checkpoint buffer too small (" + std::to_string(need) + " bytes)");
    CheckpointHeader h{kCkpMagic, c->prob.nx, c->prob.ny, c->prob.nz, c->prob.precision, c->R, c->n_patch,
                       c->A.nnz, c->t, c->prob.max_steps, c->n_pdet, 0};
    char *p = static_cast<char *>(host_buf);
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    for (int r = 0; r < c->R; ++r) {
        drts_status st = drts_read_state(c, r, reinterpret_cast<double *>(p));
        if (st != DRTS_OK) return st;
        p += c->n_states * 8;
    }
    cudaError_t e = cudaMemcpy(p, c->ledger, sizeof(double) * 4 * c->R, cudaMemcpyDeviceToHost);
    p += 4 * 8 * c->R;
    for (int r = 0; r < c->R && e == cudaSuccess && c->det && c->t > 0; ++r) {
        e = cudaMemcpy(p, c->det + size_t(r) * c->prob.max_steps * c->n_patch, sizeof(double) * c->t * c->n_patch,
                       cudaMemcpyDeviceToHost);
        p += c->t * c->n_patch * 8;
    }
    for (int r = 0; r < c->R && e == cudaSuccess && c->n_pdet > 0 && c->t > 0; ++r) {
        e = cudaMemcpy(p, c->d_pdet_hist + size_t(r) * c->prob.max_steps * c->n_pdet,
                       sizeof(double) * c->t * c->n_pdet, cudaMemcpyDeviceToHost);
        p += c->t * c->n_pdet * 8;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint_save");
    return DRTS_OK;
} catch (...) {
    return caught(c, "drts_checkpoint_save");
}

drts_status drts_checkpoint_load(drts_ctx *c, const void *host_buf, int64_t size)
try {
    NvtxRange nvtx("drts_checkpoint_load");
    if (!c || !host_buf || size < int64_t(sizeof(CheckpointHeader))) return DRTS_EINVAL;
    CheckpointHeader h;
    std::memcpy(&h, host_buf, sizeof(h));
    if (h.magic != kCkpMagic) return fail(c, DRTS_EINVAL, "not a DRTS checkpoint");
    if (h.nx != c->prob.nx || h.ny != c->prob.ny || h.nz != c->prob.nz || h.precision != c->prob.precision ||
        h.n_rhs != c->R || h.n_patch != c->n_patch || h.nnz != c->A.nnz)
        return fail(c, DRTS_EINVAL, "checkpoint is of another problem");
    if (h.n_pdet != c->n_pdet)
        return fail(c, DRTS_EINVAL, "checkpoint has another set of point detectors (set them before loading)");
    if (h.t < 0) return fail(c, DRTS_EINVAL, "checkpoint time < 0");
    if ((c->det || c->n_pdet > 0) && h.t > c->prob.max_steps)
        return fail(c, DRTS_EINVAL, "checkpoint time beyond max_steps");
    const int64_t det_steps = (c->det && h.max_steps > 0) ? h.t : 0;
    const int64_t pdet_steps = c->n_pdet > 0 ? h.t : 0;
    const int64_t need = int64_t(sizeof(h)) + int64_t(c->R) * (c->n_states * 8 + 32) +
                         int64_t(c->R) * det_steps * c->n_patch * 8 + int64_t(c->R) * pdet_steps * c->n_pdet * 8;
    if (size < need) return fail(c, DRTS_EINVAL, "checkpoint truncated");
    if ((c->t ^ h.t) & 1) std::swap(c->x, c->y);   // keep the state buffer parity of an uninterrupted run
    c->t = h.t;
    const char *p = static_cast<const char *>(host_buf) + sizeof(h);
    for (int r = 0; r < c->R; ++r) {
        drts_status st = drts_write_state(c, r, reinterpret_cast<const double *>(p));
        if (st != DRTS_OK) return st;
        p += c->n_states * 8;
    }
    cudaError_t e = cudaMemcpy(c->ledger, p, sizeof(double) * 4 * c->R, cudaMemcpyHostToDevice);
    p += 32 * c->R;
    for (int r = 0; r < c->R && e == cudaSuccess && det_steps > 0; ++r) {
        e = cudaMemcpy(c->det + size_t(r) * c->prob.max_steps * c->n_patch, p, sizeof(double) * det_steps * c->n_patch,
                       cudaMemcpyHostToDevice);
        p += det_steps * c->n_patch * 8;
    }
    for (int r = 0; r < c->R && e == cudaSuccess && pdet_steps > 0; ++r) {
        e = cudaMemcpy(c->d_pdet_hist + size_t(r) * c->prob.max_steps * c->n_pdet, p,
                       sizeof(double) * pdet_steps * c->n_pdet, cudaMemcpyHostToDevice);
        p += pdet_steps * c->n_pdet * 8;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint_load");
    return DRTS_OK;
} catch (...) {
    return caught(c, "drts_checkpoint_load");
}

drts_status drts_set_step_mode(drts_ctx *c, int32_t mode)
try {
    if (!c) return DRTS_EINVAL;
    if (mode == DRTS_STEP_LAUNCH) {
        c->step_mode = mode;
        return DRTS_OK;
    }
    if (mode == DRTS_STEP_PERSISTENT) {
        if (c->R != 1) return fail(c, DRTS_EUNSUPPORTED, "persistent mode steps one right-hand side");
        if (c->n_bulk_groups > 0) return fail(c, DRTS_EUNSUPPORTED, "sub-step sources need the launch step mode");
        const int blocks = persistent_blocks(c->prob.precision, c->threads, 1);
        if (blocks < 1) return fail(c, DRTS_EUNSUPPORTED, "cooperative launch not available");
        c->step_mode = mode;
        return DRTS_OK;
    }
    return fail(c, DRTS_EINVAL, "unknown step mode");
} catch (...) {
    return caught(c, "drts_set_step_mode");
}

drts_status drts_set_fault(drts_ctx *c, int32_t kind, int64_t arg)
try {
    if (!c) return DRTS_EINVAL;
    switch (kind) {
    case DRTS_FAULT_NONE:
        c->fault_skip_chunk = -1;
        c->fault_skip_barrier = 0;
        c->spin_limit = 1u << 22;
        return DRTS_OK;
    case DRTS_FAULT_SKIP_BARRIER:
        if (c->step_mode != DRTS_STEP_PERSISTENT) return fail(c, DRTS_ESTATE, "no grid barrier outside persistent mode");
        c->fault_skip_barrier = 1;
        return DRTS_OK;
    case DRTS_FAULT_SKIP_COPY:
        if (arg < 0) return fail(c, DRTS_EINVAL, "chunk index must be >= 0");
        if (c->R != 1 || c->variant < 3 || c->variant > 6)
            return fail(c, DRTS_ESTATE, "only the bulk-copy step variants (3-6) have copies to skip");
        c->fault_skip_chunk = arg;
        return DRTS_OK;
    case DRTS_FAULT_SPIN_LIMIT:
        if (arg < 1 || arg > (int64_t(1) << 30)) return fail(c, DRTS_EINVAL, "spin limit must be 1..2^30");
        c->spin_limit = uint32_t(arg);
        return DRTS_OK;
    default:
        return fail(c, DRTS_EINVAL, "unknown fault kind");
    }
} catch (...) {
    return caught(c, "drts_set_fault");
}

drts_status drts_set_allocator(drts_alloc_fn alloc_fn, drts_free_fn free_fn, void *user)
{
    if (!alloc_fn != !free_fn) return DRTS_EINVAL;
    std::lock_guard<std::mutex> lock(g_allocator_mu);
    g_allocator = Allocator{alloc_fn, free_fn, alloc_fn ? user : nullptr};
    return DRTS_OK;
}

drts_status drts_set_alloc_fault(int64_t n_ok)
{
    g_alloc_fault.store(n_ok < 0 ? -1 : n_ok);
    return DRTS_OK;
}

drts_status drts_state_sum_noalloc(drts_ctx *c, int32_t rhs, double *out_device)
try {
    if (!c) return DRTS_EINVAL;
    if (rhs < 0 || rhs >= c->R || !out_device) return fail(c, DRTS_EINVAL, "bad arguments");
    if (c->tc) return fail(c, DRTS_EUNSUPPORTED, "not available for the tensor-core state layout");
    if (c->n_states > noalloc_max_states())
        return fail(c, DRTS_EINVAL, "state vector of " + std::to_string(c->n_states) +
                                        " states exceeds the static scratch limit of " +
                                        std::to_string(noalloc_max_states()));
    cudaError_t e = launch_state_sum_noalloc(rhs_view(c, c->x, rhs).base, c->prob.precision, c->n_states,
                                             rhs_view(c, c->x, rhs).stride, 0, out_device,
                                             c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "state_sum_noalloc");
    return DRTS_OK;
} catch (...) {
    return caught(c, "drts_state_sum_noalloc");
}

namespace {

// Column `state` of the matrix built for the path fraction frac (Eq. 18/19/21
// with the path frac * L_k, folded like the system matrix), as (target
// state, value) pairs in ascending state order, and the mass that leaves the
// grid.  Synchronous.
drts_status source_column_host(drts_ctx *c, int64_t state, double frac,
                               std::vector<std::pair<int64_t, double>> &col, double *exit_mass)
{
    HostTables tf;
    drts_problem p = c->prob;
    p.media = c->media.data();
    p.interface = DRTS_INTERFACE_FIRST_ORDER;   // sub-step columns use the first-order fold
    const std::string terr = build_host_tables(p, tf, frac);
    if (!terr.empty()) return fail(c, DRTS_EINVAL, terr);
    double *dW = nullptr, *dout = nullptr;
    std::vector<double> out(size_t(kOffs) * kDirs, 0.0);
    cudaError_t e = cudaMalloc(&dW, tf.W.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dout, out.size() * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dW, tf.W.data(), tf.W.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    DevTables Tf = c->T;
    Tf.W = dW;
    Tf.interface = DRTS_INTERFACE_FIRST_ORDER;
    if (e == cudaSuccess) e = launch_source_column(Tf, state, dout, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out.data(), dout, out.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (dW) cudaFree(dW);
    if (dout) cudaFree(dout);
    if (e != cudaSuccess) return cuda_fail(c, e, "source column");
    const int nx = c->prob.nx, ny = c->prob.ny, nz = c->prob.nz;
    const int64_t v = state / kDirs;
    const int n = int(state % kDirs);
    const int x = int(v % nx), y = int(v / nx % ny), z = int(v / (int64_t(nx) * ny));
    col.clear();
    for (int g = 0; g < kOffs * kDirs; ++g) {
        if (!(out[g] > 0.0)) continue;
        const int d = g / kDirs, m = g % kDirs;
        const int64_t vj = (int64_t(z + d / 9 - 1) * ny + (y + d / 3 % 3 - 1)) * nx + (x + d % 3 - 1);
        col.emplace_back(vj * kDirs + m, out[g]);
    }
    if (exit_mass) {
        const int bx = x == 0 ? 0 : (x == nx - 1 ? 2 : 1);
        const int by = y == 0 ? 0 : (y == ny - 1 ? 2 : 1);
        const int bz = z == 0 ? 0 : (z == nz - 1 ? 2 : 1);
        const int k = c->med_host[size_t(v)];
        *exit_mass = tf.exit_total[(size_t(k) * 27 + bz * 9 + by * 3 + bx) * kDirs + n];
    }
    return DRTS_OK;
}

// Flatten every rhs's sub-step source into (state, rhs) groups and upload.
drts_status upload_bulk(drts_ctx *c)
{
    std::vector<BulkGroup> groups;
    std::vector<int32_t> rhs_off(size_t(c->R) + 1, 0);
    std::vector<BulkEntry> entries;
    std::vector<SourceProfile> prof;
    std::vector<double> vals;
    struct Trip { int64_t state; double w; int32_t prof; };
    for (int r = 0; r < c->R; ++r) {
        rhs_off[r] = int32_t(groups.size());
        const drts_ctx::SubstepSource &ss = c->substep[r];
        if (ss.state.empty() || ss.n_t == 0) continue;
        const int32_t prof0 = int32_t(prof.size());
        for (int j = 0; j < ss.n_sub; ++j) {
            prof.push_back(SourceProfile{ss.t0, ss.n_t, int32_t(vals.size()), 0, 0});
            for (int32_t t = 0; t < ss.n_t; ++t) vals.push_back(ss.profile[size_t(t) * ss.n_sub + j]);
        }
        std::vector<Trip> tr;
        for (size_t i = 0; i < ss.state.size(); ++i)
            for (int j = 0; j < ss.n_sub; ++j)
                for (const auto &pv : ss.columns[i * ss.n_sub + j])
                    tr.push_back(Trip{pv.first, ss.weight[i] * pv.second, prof0 + j});
        std::stable_sort(tr.begin(), tr.end(), [](const Trip &a, const Trip &b) { return a.state < b.state; });
        for (size_t q = 0; q < tr.size();) {
            BulkGroup g{tr[q].state, r, int32_t(entries.size()), 0, 0};
            for (; q < tr.size() && tr[q].state == g.state; ++q) {
                entries.push_back(BulkEntry{tr[q].w, tr[q].prof, 0});
                ++g.count;
            }
            groups.push_back(g);
        }
    }
    rhs_off[c->R] = int32_t(groups.size());
    if (entries.size() > size_t(1) << 30) return fail(c, DRTS_EINVAL, "too many sub-step source entries");
    cudaError_t e = cudaSuccess;
    drelease(c, c->d_bulk_groups);          // the previous set (if any)
    drelease(c, c->d_bulk_rhs_off);
    drelease(c, c->d_bulk_entries);
    drelease(c, c->d_bulk_prof);
    drelease(c, c->d_bulk_prof_vals);
    c->n_bulk_groups = 0;
    if (!groups.empty()) {
        if ((e = upload(c, &c->d_bulk_groups, groups)) != cudaSuccess ||
            (e = upload(c, &c->d_bulk_rhs_off, rhs_off)) != cudaSuccess ||
            (e = upload(c, &c->d_bulk_entries, entries)) != cudaSuccess ||
            (e = upload(c, &c->d_bulk_prof, prof)) != cudaSuccess ||
            (e = upload(c, &c->d_bulk_prof_vals, vals)) != cudaSuccess)
            return cuda_fail(c, e, "sub-step source upload");
    }
    c->n_bulk_groups = int(groups.size());
    return sync_check(c, "sub-step source upload");
}

}  // namespace

drts_status drts_source_column(drts_ctx *c, int64_t state_idx, double frac, int32_t cap, int64_t *out_state,
                               double *out_value, int32_t *count, double *exit_mass)
try {
    if (!c) return DRTS_EINVAL;
    if (state_idx < 0 || state_idx >= c->n_states) return fail(c, DRTS_EINVAL, "state out of range");
    if (!(frac > 0.0 && frac <= 1.0)) return fail(c, DRTS_EINVAL, "frac must be in (0, 1]");
    if (!count || cap < 0 || (cap > 0 && (!out_state || !out_value)))
        return fail(c, DRTS_EINVAL, "bad output arrays");
    std::vector<std::pair<int64_t, double>> col;
    drts_status st = source_column_host(c, state_idx, frac, col, exit_mass);
    if (st != DRTS_OK) return st;
    *count = int32_t(col.size());
    if (int64_t(col.size()) > cap)
        return fail(c, DRTS_EINVAL, "cap too small (" + std::to_string(col.size()) + " entries)");
    for (size_t i = 0; i < col.size(); ++i) {
        out_state[i] = col[i].first;
        out_value[i] = col[i].second;
    }
    return DRTS_OK;
} catch (...) {
    return caught(c, "drts_source_column");
}

drts_status drts_inject_source_substeps(drts_ctx *c, int32_t rhs, int32_t n_entries, const int64_t *state_idx,
                                        const double *weight, int32_t n_sub, int64_t t0, int32_t n_t,
                                        const double *profile)
try {
    if (!c) return DRTS_EINVAL;
    if (rhs < 0 || rhs >= c->R) return fail(c, DRTS_EINVAL, "rhs out of range");
    if (n_entries < 0 || n_entries > kMaxSrc) return fail(c, DRTS_EINVAL, "n_entries must be 0..64");
    if (n_sub < 1 || n_sub > 64) return fail(c, DRTS_EINVAL, "n_sub must be 1..64");
    if (n_t < 0 || (n_t > 0 && n_entries > 0 && !profile)) return fail(c, DRTS_EINVAL, "bad profile");
    if (c->tc && n_entries > 0)
        return fail(c, DRTS_EUNSUPPORTED, "sub-step sources are not available with the tensor-core batched step");
    if (n_entries > 0 && (!state_idx || !weight)) return fail(c, DRTS_EINVAL, "NULL source arrays");
    drts_ctx::SubstepSource ss;
    const int ns = n_sub;
    for (int i = 0; i < n_entries; ++i) {
        if (state_idx[i] < 0 || state_idx[i] >= c->n_states) return fail(c, DRTS_EINVAL, "source state out of range");
        if (!std::isfinite(weight[i])) return fail(c, DRTS_EINVAL, "source weight not finite");
    }
    if (n_entries > 0 && n_t > 0) {
        for (int64_t q = 0; q < int64_t(n_t) * ns; ++q)
            if (!std::isfinite(profile[q])) return fail(c, DRTS_EINVAL, "profile value not finite");
        ss.state.assign(state_idx, state_idx + n_entries);
        ss.weight.assign(weight, weight + n_entries);
        ss.n_sub = ns;
        ss.t0 = t0;
        ss.n_t = n_t;
        ss.profile.assign(profile, profile + int64_t(n_t) * ns);
        for (int i = 0; i < n_entries; ++i)
            for (int j = 0; j < ns; ++j) {
                // sub-interval j, taken at its midpoint: the rest of the step is frac of the path
                const double frac = 1.0 - (j + 0.5) / ns;
                std::vector<std::pair<int64_t, double>> col;
                drts_status st = source_column_host(c, state_idx[i], frac, col, nullptr);
                if (st != DRTS_OK) return st;
                ss.columns.push_back(std::move(col));
            }
    }
    c->substep[rhs] = std::move(ss);
    return upload_bulk(c);
} catch (...) {
    return caught(c, "drts_inject_source_substeps");
}

drts_status drts_substep_count(drts_ctx *c, int64_t state_idx, int32_t *n_sub)
try {
    if (!c || !n_sub) return DRTS_EINVAL;
    if (state_idx < 0 || state_idx >= c->n_states) return fail(c, DRTS_EINVAL, "state out of range");
    // sub-intervals of dr / c: the path L_k in half voxels (2 dr = h), rounded up
    const int k = c->med_host[size_t(state_idx / kDirs)];
    *n_sub = std::max(1, int(std::ceil(2.0 * c->host.lam[k] - 1e-9)));
    return DRTS_OK;
} catch (...) {
    return caught(c, "drts_substep_count");
}

drts_status drts_set_point_detectors(drts_ctx *c, int32_t n_det, int64_t n_entries, const int32_t *det,
                                     const int64_t *state_idx, const double *weight)
try {
    if (!c) return DRTS_EINVAL;
    if (n_det < 0 || n_det > 65535) return fail(c, DRTS_EINVAL, "n_det must be 0..65535");
    if (n_entries < 0 || (n_entries > 0 && (!det || !state_idx || !weight)))
        return fail(c, DRTS_EINVAL, "bad entry arrays");
    auto drop_old = [&]() {                 // the previous set (if any) goes
        c->n_pdet = 0;
        drelease(c, c->d_pdet_off);
        drelease(c, c->d_pdet_state);
        drelease(c, c->d_pdet_w);
        drelease(c, c->d_pdet_hist);
    };
    if (n_det == 0) {
        drop_old();
        return DRTS_OK;
    }
    if (c->prob.max_steps <= 0)
        return fail(c, DRTS_ESTATE, "point detectors keep a history: max_steps must be > 0");
    if (c->t > c->prob.max_steps) return fail(c, DRTS_ESTATE, "t is beyond max_steps");
    std::vector<int64_t> off(size_t(n_det) + 1, 0);
    for (int64_t e = 0; e < n_entries; ++e) {
        if (det[e] < 0 || det[e] >= n_det) return fail(c, DRTS_EINVAL, "detector index out of range");
        if (state_idx[e] < 0 || state_idx[e] >= c->n_states) return fail(c, DRTS_EINVAL, "state out of range");
        if (!std::isfinite(weight[e])) return fail(c, DRTS_EINVAL, "weight not finite");
        ++off[size_t(det[e]) + 1];
    }
    for (int d = 0; d < n_det; ++d) off[d + 1] += off[d];
    std::vector<int64_t> st(static_cast<size_t>(n_entries));
    std::vector<double> w(static_cast<size_t>(n_entries));
    std::vector<int64_t> pos(off.begin(), off.end() - 1);
    for (int64_t e = 0; e < n_entries; ++e) {      // grouped by detector, entry order kept
        const int64_t q = pos[det[e]]++;
        st[q] = state_idx[e];
        w[q] = weight[e];
    }
    drop_old();
    cudaError_t e = cudaSuccess;
    if ((e = upload(c, &c->d_pdet_off, off)) != cudaSuccess || (e = upload(c, &c->d_pdet_state, st)) != cudaSuccess ||
        (e = upload(c, &c->d_pdet_w, w)) != cudaSuccess ||
        (e = dalloc(c, &c->d_pdet_hist, sizeof(double) * size_t(c->R) * c->prob.max_steps * n_det)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->d_pdet_hist, 0, sizeof(double) * size_t(c->R) * c->prob.max_steps * n_det,
                             c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "point detector upload");
    c->n_pdet = n_det;
    return sync_check(c, "point detector upload");
} catch (...) {
    return caught(c, "drts_set_point_detectors");
}

drts_status drts_read_point_detectors(drts_ctx *c, int32_t rhs, int64_t t_begin, int64_t t_end, double *host_out)
try {
    if (!c) return DRTS_EINVAL;
    if (rhs < 0 || rhs >= c->R) return fail(c, DRTS_EINVAL, "rhs out of range");
    if (c->n_pdet <= 0) return fail(c, DRTS_ESTATE, "no point detectors set");
    if (t_begin < 0 || t_end < t_begin || t_end > std::min(c->t, c->prob.max_steps))
        return fail(c, DRTS_EINVAL, "bad step range");
    if (t_end == t_begin) return DRTS_OK;
    if (!host_out) return fail(c, DRTS_EINVAL, "host_out is NULL");
    cudaError_t e = cudaMemcpyAsync(host_out, c->d_pdet_hist + (size_t(rhs) * c->prob.max_steps + t_begin) * c->n_pdet,
                                    sizeof(double) * (t_end - t_begin) * c->n_pdet, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "read_point_detectors");
    return sync_check(c, "read_point_detectors");
} catch (...) {
    return caught(c, "drts_read_point_detectors");
}

drts_status drts_sensor_response(drts_ctx *c, int32_t rhs, int32_t which, int64_t t_begin, int64_t t_end, int32_t w,
                                 const double *h, double *host_out)
try {
    if (!c) return DRTS_EINVAL;
    if (rhs < 0 || rhs >= c->R) return fail(c, DRTS_EINVAL, "rhs out of range");
    if (w < 0 || w > (1 << 20) || !h) return fail(c, DRTS_EINVAL, "w must be 0..2^20 and h non-NULL");
    const double *D = nullptr;
    int n_det = 0;
    if (which == DRTS_SENSOR_FACE) {
        if (!c->det || c->n_patch <= 0) return fail(c, DRTS_ESTATE, "no face detector history");
        D = c->det + size_t(rhs) * c->prob.max_steps * c->n_patch;
        n_det = c->n_patch;
    } else if (which == DRTS_SENSOR_POINT) {
        if (c->n_pdet <= 0) return fail(c, DRTS_ESTATE, "no point detectors set");
        D = c->d_pdet_hist + size_t(rhs) * c->prob.max_steps * c->n_pdet;
        n_det = c->n_pdet;
    } else {
        return fail(c, DRTS_EINVAL, "which must be DRTS_SENSOR_FACE or DRTS_SENSOR_POINT");
    }
    const int64_t t_rec = std::min(c->t, c->prob.max_steps);
    if (t_begin < 0 || t_end < t_begin || t_end > t_rec) return fail(c, DRTS_EINVAL, "bad step range");
    if (t_end == t_begin) return DRTS_OK;
    if (!host_out) return fail(c, DRTS_EINVAL, "host_out is NULL");
    double *dh = nullptr, *dm = nullptr;
    const size_t nm = size_t(t_end - t_begin) * n_det;
    cudaError_t e = cudaMallocAsync(&dh, sizeof(double) * (2 * size_t(w) + 1), c->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&dm, sizeof(double) * nm, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dh, h, sizeof(double) * (2 * size_t(w) + 1), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_sensor_response(D, t_rec, n_det, t_begin, t_end, w, dh, dm, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, dm, sizeof(double) * nm, cudaMemcpyDeviceToHost, c->stream);
    if (dh) cudaFreeAsync(dh, c->stream);
    if (dm) cudaFreeAsync(dm, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "sensor_response");
    return sync_check(c, "sensor_response");
} catch (...) {
    return caught(c, "drts_sensor_response");
}

void drts_destroy(drts_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (const DevBuffer &b : c->allocs) free_buffer(b, c->stream);
    delete c;
}

const char *drts_last_error(const drts_ctx *c)
{
    return c ? c->err.c_str() : g_assemble_error.c_str();
}

}  // extern "C"
