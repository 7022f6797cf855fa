// Device-side data of an assembled DRTS problem and the launch wrappers the
// C ABI calls.  All kernels target sm_103a.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "drts_internal.h"

namespace drts {

// Lookup tables the device assembler reads (uploaded once per problem).
struct DevTables {
    int nx, ny, nz;
    int64_t V;                  // voxels
    int K;                      // media
    const double *W;            // [K][26][27][26] raw stencil
    const int32_t *tmpl_off;    // [K][26][28]
    const uint8_t *tmpl_n;
    const double *tmpl_val;
    const double *r_edge;       // [K][4]
    const double *r_int;        // [K][K][4]
    const double *nref;         // [K]
    const uint8_t *med;         // [V] medium of each voxel
    const uint8_t *plain;       // [V] 1 when the voxel's rows need no folding
    const float *dir_scale;     // [26] FP16 tier row scale by direction (or null)
    // planar two-step interface crossing (DRTS_INTERFACE_TWO_STEP; else 0 / null)
    int interface;
    const int32_t *pair_slot;   // [K][K] slot of (source medium, medium of the next z layer), or -1
    const uint8_t *cross;       // [P][26] direction n reaches the plane within the step
    const double *W2f;          // [P][26][27][26] crossing entries folded at edges and interfaces
    const double *W2n;          // [P][26][27][26] crossing entries folded at the grid edge only
};

// Sliced storage of A: slice q = voxel block b (32 voxels) * 26 + direction
// m; lane l of the slice is row (voxel 32b+l, direction m).  Entry e of a row
// sits at ((slice_ptr[q] + e/4) * 32 + lane) * 4 + e%4 (lane-interleaved
// groups of four), so one warp-wide 16-byte load per lane moves 128 entries.
struct SlicedMatrix {
    int precision = DRTS_FP32;
    int64_t n_slices = 0;
    int64_t n_groups = 0;       // sum of slice_len4 (units of 32 lanes x 4)
    int64_t nnz = 0;
    int64_t nnz_stored = 0;     // nnz + second FP16 terms of split values
    void *vals = nullptr;       // double / float / __half [n_groups*128]
    uint16_t *codes = nullptr;  // [n_groups*128] offset_index*26 + n
    float *row_scale = nullptr; // FP16 tier: [n_slices*32]
    int64_t *slice_ptr = nullptr;   // [n_slices] in groups
    int32_t *slice_len4 = nullptr;  // [n_slices]
    int32_t *row_len = nullptr;     // [n_slices*32]
};

struct SourceEntry {
    int32_t slice;     // slice holding the target state
    int32_t lane;      // lane (row) within it
    int32_t rhs;
    int32_t prof;      // index of the rhs profile
    double w;          // weight
};

struct SourceProfile {
    int64_t t0;
    int32_t n_t;
    int32_t off;       // offset into the profile value array
    int32_t pad0, pad1;
};

// Column functionals of one step (per ledger class / face mask / direction;
// the class of a voxel is its medium, or with two-step interfaces the class
// of its z layer).
struct StepTables {
    const double *absorb;      // [C] absorbed fraction of a state
    const double *absorb_dir;  // [C][26] per direction, or null when absorb[C] holds for all
    const double *exit_total;  // [C][27][26]
    const double *exit_det;    // [C][27][26]
};

// Sparse detector rows F of Eq. 27 (point detectors): the entries of
// detector d are off[d] .. off[d+1], each a canonical state and a weight.
struct PointDetectors {
    int n_det;
    const int64_t *off;        // [n_det + 1]
    const int64_t *state;      // canonical state of each entry
    const double *w;
    double *hist;              // [r][max_steps][n_det] readout history, or null
    int64_t stride_r;          // max_steps * n_det
};

// Sub-step sources (Section 4.1 time partition of the source term): groups of
// entries that land on one (state, rhs); group g adds
// sum_e w_e P_{prof_e}(t) to y[state] after the product.
struct BulkGroup {
    int64_t state;
    int32_t rhs;
    int32_t first;             // entries first .. first + count - 1
    int32_t count;
    int32_t pad;
};
struct BulkEntry {
    double w;
    int32_t prof;              // index into the sub-step profiles
    int32_t pad;
};
struct BulkSources {
    int n_groups;
    const BulkGroup *groups;   // sorted by (rhs, state)
    const int32_t *rhs_off;    // [R + 1] group range of each rhs
    const BulkEntry *entries;
    const SourceProfile *prof;
    const double *prof_vals;
};

// Tensor-core batched step: A stored union-dense (per voxel, per block role
// d, the values at the role's fixed (n, m) positions).  Voxel j's data is
// voxel_bytes long; role d's chunk at chunk_off[d] holds three fp16 arrays
// (a0, a1, a2) of the role's padded position count followed by 32 bytes of
// row exponents (Ea + 160 per direction m).
struct TcPlan {
    int role_off[28];           // role d owns positions [role_off[d], role_off[d+1]) (multiples of 8)
    int chunk_off[28];          // byte offset of role d's chunk within a voxel
    int64_t voxel_bytes;        // bytes per voxel (multiple of 16)
    const uint16_t *pos;        // [role_off[27]] (n << 8) | m; padding entries (31 << 8)
    const void *Au;             // [V][voxel_bytes]
};

struct StepArgs {
    SlicedMatrix A;
    int nx, ny, nz;
    int64_t V;
    int R;                     // right-hand sides
    int64_t rhs_stride;        // elements between right-hand sides of a state buffer
    const void *x;             // state at t, layout [r*rhs_stride + n*V + v]
    void *y;                   // state at t+1
    const uint8_t *cls;        // [V] ledger class of each voxel (StepTables)
    StepTables tab;
    int det_face, det_nu, det_nv, n_patch;
    double *det;               // det[r][t_hist][patch] base, or null
    int64_t det_stride_r;      // elements between rhs
    int64_t t;                 // time index of x
    double *ledger;            // [R][4]: sum x, injected, absorbed, exited
    int n_src;
    const SourceEntry *src;
    const SourceProfile *prof; // [R]
    const double *prof_vals;
    const double *step_scale;  // [R] host-supplied source factors of this step, or null
    int rhs_tile;
    int *err;                  // set to 1 when a bounded device wait gives up
    TcPlan tcp;                // tensor-core batched step: union-dense A
    const uint8_t *src_voxel;  // [V] 1 where some source entry targets the voxel
    uint32_t spin_limit;       // polls before a device wait gives up
    int64_t fault_skip_chunk;  // tests only: chunk warp 0 never copies (-1 none)
    int tcx;                   // 1: tensor-core state layout (8 KB fp16 (x0, x1, Ex) tile per voxel)
    PointDetectors pd;         // point detectors read from x (n_det = 0: none)
    BulkSources bulk;          // sub-step sources added to y (n_groups = 0: none)
};

// assembler (drts_assemble.cu)
cudaError_t launch_classify(const DevTables &T, uint8_t *plain, cudaStream_t s);
cudaError_t launch_count(const DevTables &T, SlicedMatrix &A, unsigned long long *n_split, cudaStream_t s);
cudaError_t launch_scan(SlicedMatrix &A, int64_t *d_total, cudaStream_t s);
cudaError_t launch_fill(const DevTables &T, SlicedMatrix &A, cudaStream_t s);
cudaError_t launch_export(const SlicedMatrix &A, int nx, int ny, int nz, int64_t row_begin,
                          int64_t row_end, const int64_t *d_row_ptr, int32_t *d_col,
                          double *d_val, cudaStream_t s);
cudaError_t launch_count_export(const SlicedMatrix &A, int64_t V, int64_t row_begin,
                                int64_t row_end, int64_t *d_counts, cudaStream_t s);

// step (drts_step.cu)
// variant: 0-2 registers path (prefetch depth 1-3), 3-6 bulk-copy paths
// (shared-memory stages of (G, S) = (8,3), (4,3), (4,4), (2,6)), 7-8
// shared-memory x-halo paths with 13 or 26 warps (nx a multiple of 32), 9
// registers path with matrix and gather streams both pipelined, 10-11 two
// or four warps per slice (small grids), 12-13 registers path with 32-bit
// indices held to six or eight CTAs per SM, 14 eight warps per slice
cudaError_t launch_step(const StepArgs &a, int variant, int blocks, int threads, cudaStream_t s);
int step_default_blocks(int precision, int R, int threads, int variant);
constexpr int kStepVariants = 15;
// persistent multi-step kernel (cooperative launch, bounded grid barrier);
// split = warps per slice (1, 2, 4 or 8)
int persistent_blocks(int precision, int threads, int split);
cudaError_t launch_persistent(const StepArgs &a, void *other, int64_t n_steps, double *det_base, int64_t max_steps,
                              unsigned *bar, int fault_skip_barrier, int blocks, int threads, int split,
                              cudaStream_t s);
cudaError_t launch_to_canonical(const void *x, int precision, int64_t V, int R, int r,
                                double *out, cudaStream_t s);
cudaError_t launch_from_canonical(const double *in, int precision, int64_t V, int R, int r,
                                  void *x, cudaStream_t s);
cudaError_t launch_ledger_sum(const void *x, int precision, int64_t n, int R, int r,
                              double *out, cudaStream_t s);

// batched step (drts_batched.cu): functionals (detector + ledger of X(t))
// when asked, then ceil(R / rhs_tile) passes of the product over A; order 0
// strides warps over slices, order 1 is block-major, order 2 stages each
// voxel block's x halo in shared memory (one launch, fixed tile and block
// shape: 26 warps, 4 FP32 / 2 FP64 right-hand sides per pass)
constexpr int kBatchedOrders = 3;
int batched_blocks_per_sm(int precision, int rhs_tile, int threads, int order);
cudaError_t launch_batched_step(const StepArgs &a, int n_rhs, int rhs_tile, int order, int blocks, int threads,
                                bool functionals, cudaStream_t s);

// tensor-core batched step (drts_tensor.cu): state tile per voxel of 64
// right-hand sides of x0 and x1 (bf16, 8 KB); flags / convert build the
// union-dense A from the sliced FP32 matrix
size_t tcx_state_bytes(int64_t V);
int tc_stage_limit();
int tc_position_limit();
int tc_blocks_per_sm(std::string *why);
cudaError_t launch_tc_flags(const SlicedMatrix &A, int64_t V, uint8_t *flags, cudaStream_t s);
cudaError_t launch_tc_convert(const SlicedMatrix &A, int64_t V, const int16_t *pidx, const TcPlan &P,
                              void *Au, cudaStream_t s);
cudaError_t launch_tc_step(const StepArgs &a, bool functionals, cudaStream_t s);
cudaError_t launch_tc_to_canonical(const void *x, int64_t V, int r, double *out, cudaStream_t s);
cudaError_t launch_tc_from_canonical(const double *in, int64_t V, int r, void *x, cudaStream_t s);
cudaError_t launch_tc_sum(const void *x, int64_t V, int r, double *out, cudaStream_t s);

// Eq. 26/27 extensions (drts_functionals.cu): point detectors of x(t) (one
// CTA per detector and rhs), sub-step sources added to y(t+1), and the
// sensor response of a detector history
cudaError_t launch_point_detectors(const StepArgs &a, cudaStream_t s);
cudaError_t launch_bulk_sources(const StepArgs &a, cudaStream_t s);
cudaError_t launch_sensor_response(const double *D, int64_t t_rec, int n_det, int64_t t_begin, int64_t t_end,
                                   int w, const double *h, double *M, cudaStream_t s);
// column (state) of the system matrix built with a partial path (tables Tf):
// out[d*26 + m] = mass reaching (voxel + offset d, direction m), 0 off the grid
cudaError_t launch_source_column(const DevTables &Tf, int64_t state, double *out, cudaStream_t s);

// no-allocation state sum (drts_noalloc.cu)
int64_t noalloc_max_states();
cudaError_t launch_state_sum_noalloc(const void *x, int precision, int64_t n, int R, int r,
                                     double *out, cudaStream_t s);

}  // namespace drts
