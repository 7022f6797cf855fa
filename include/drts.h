/*
 * drts.h - C ABI of the GB300 DRTS library (libdrts.so).
 *
 * The Dynamic Radiative Transfer System (Georgakopoulos, Politopoulos and
 * Georgiou, arXiv:1611.08536) advances photon populations J(X_i, S_n) over
 * (voxel, direction) states with one sparse matrix-vector product per time
 * step, J(t+dt) = A J(t) + B P(t) (Eq. 26).  A is assembled once (Eq. 18-23,
 * Section 3) and stays resident on the GPU; every step runs in the library's
 * CUDA kernels.
 *
 * Geometry and state order (Eq. 22):
 *   cubic grid nx*ny*nz, voxel v = (z*ny + y)*nx + x, voxel size h = 2dr;
 *   26 lattice directions d enumerating {-1,0,1}^3 \ {0}, dz slowest, dx
 *   fastest; canonical state index s = v*26 + d.
 *   dt = h / c_max: medium k moves light L_k = h * n_min / n_k per step.
 *
 * Conventions shared by every call:
 *   - Every call returns a drts_status; nothing aborts or traps.  After an
 *     error, drts_last_error(ctx) describes it.  No C++ exception leaves the
 *     library: a host allocation that fails inside a call is DRTS_ENOMEM
 *     (the call's partial work on a new context is freed).
 *   - Caller-owned host inputs are copied during the call; the context owns
 *     all device memory it allocates and frees it in drts_destroy.
 *   - Work is queued on the CUDA stream given to drts_assemble (NULL = the
 *     default stream).  drts_step_n returns before the GPU finishes; the
 *     read_* calls synchronise that stream.
 *   - A context is not thread-safe; separate contexts are independent.
 *   - Sticky CUDA errors surface as DRTS_ECUDA; a device-side wait that
 *     runs out of its iteration budget surfaces as DRTS_ETIMEOUT.
 */
#ifndef DRTS_H
#define DRTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t drts_status;
#define DRTS_OK 0
#define DRTS_EINVAL 1        /* bad argument or problem description */
#define DRTS_ENOMEM 2        /* device or host allocation failed */
#define DRTS_ECUDA 3         /* CUDA runtime error (sticky or launch) */
#define DRTS_ETIMEOUT 4      /* a bounded device-side wait gave up */
#define DRTS_ESTATE 5        /* call not valid in the context's state */
#define DRTS_EUNSUPPORTED 6  /* valid request this build does not support */

/* boundary treatment of the grid edge (Section 4.2 readings) */
#define DRTS_OPEN 0          /* mass reaching outside the grid leaves */
#define DRTS_MIRROR 1        /* mass is reflected back (closed box) */
#define DRTS_FRESNEL 2       /* unpolarised Fresnel split against n_outside */

/* treatment of a change of refractive index inside the grid (Section 4.2) */
#define DRTS_INTERFACE_FIRST_ORDER 0  /* each raw target folded once: the Fresnel share at
                                         the lattice direction's angle is reflected, the rest
                                         transmitted without a change of direction; the step
                                         keeps the source medium throughout */
#define DRTS_INTERFACE_TWO_STEP 1     /* planar interfaces normal to z (one medium per z
                                         layer): a state whose direction reaches the plane
                                         half a voxel away within the step travels in two
                                         parts, splitting at the crossing point into the
                                         Fresnel share reflected at the true incidence angle
                                         and the share refracted by Snell's law, which
                                         finishes the step in the other medium at its speed */

/* weights of the outgoing lattice directions in the discrete
 * Henyey-Greenstein kernel (Section 2, the scattering kernel g(S, S') on the
 * partition of directions of Section 3):
 *   DRTS_HG_EQUAL       G[n][m] = p(S_n . S_m) / sum_m' p(S_n . S_m'): every
 *                       lattice direction counts alike (the default);
 *   DRTS_HG_QUADRATURE  each direction also weighted by its share of the
 *                       sphere, G[n][m] = w_m p(S_n . S_m) / sum_m' w_m'
 *                       p(S_n . S_m'), with w = 1/21 per axis, 4/105 per face
 *                       diagonal and 9/280 per body diagonal: the 26
 *                       directions with these weights integrate every
 *                       polynomial of degree <= 7 on the sphere exactly, so
 *                       the kernel's mean cosine is g up to the HG terms of
 *                       degree 7 and above.  The paper gives its directions
 *                       as quadrature points (Lebedev) without saying whether
 *                       the kernel carries their weights. */
#define DRTS_HG_EQUAL 0
#define DRTS_HG_QUADRATURE 1

/* storage / arithmetic precision of the time step */
#define DRTS_FP64 0          /* A, state and accumulation in FP64 */
#define DRTS_FP32 1          /* A and state in FP32, FP32 accumulation */
#define DRTS_FP16_ROWSCALE 2 /* A in FP16 with a per-row FP32 scale, FP32 state; a value
                                 of 512 or more times its row scale is kept as two FP16
                                 terms (hi + lo, 21 significant bits) */

/* detector faces: 2*axis + (1 for the high side) */
#define DRTS_FACE_MX 0
#define DRTS_FACE_PX 1
#define DRTS_FACE_MY 2
#define DRTS_FACE_PY 3
#define DRTS_FACE_MZ 4
#define DRTS_FACE_PZ 5
#define DRTS_FACE_NONE (-1)

/* Optical properties of one medium (Section 2): scattering coefficient
 * mu_s (1/mm, Eq. 2), absorption coefficient mu_a (1/mm, Eq. 8),
 * Henyey-Greenstein anisotropy g of the kernel g(S,S') (Section 5) and
 * refractive index n (speed c0/n, Section 4.2). */
typedef struct drts_medium {
    double mu_s, mu_a, g, n;
} drts_medium;

typedef struct drts_problem {
    int32_t nx, ny, nz;              /* grid size, each >= 2 */
    double voxel_mm;                 /* h = 2dr */
    int32_t n_media;                 /* 1..255 */
    const drts_medium *media;        /* [n_media], host, copied */
    const uint8_t *medium_of_voxel;  /* [nx*ny*nz] (x fastest), host, copied */
    double n_outside;                /* refractive index outside the grid */
    int32_t boundary;                /* DRTS_OPEN / DRTS_MIRROR / DRTS_FRESNEL */
    int32_t precision;               /* DRTS_FP64 / DRTS_FP32 / DRTS_FP16_ROWSCALE */
    int32_t n_rhs;                   /* right-hand sides stepped together, 1..64 */
    int32_t det_face;                /* detector face or DRTS_FACE_NONE */
    int32_t det_nu, det_nv;          /* detector patch grid on that face */
    int64_t max_steps;               /* detector history capacity in steps */
    int32_t batched_kernel;          /* n_rhs > 1: DRTS_BATCHED_CUDA_CORES or DRTS_BATCHED_TENSOR */
    int32_t interface;               /* DRTS_INTERFACE_FIRST_ORDER or DRTS_INTERFACE_TWO_STEP;
                                        TWO_STEP needs one medium per z layer (else
                                        DRTS_EINVAL).  Sub-step source columns
                                        (drts_source_column, drts_inject_source_substeps)
                                        use the first-order fold in both modes. */
    int32_t direction_weights;       /* DRTS_HG_EQUAL (0) or DRTS_HG_QUADRATURE */
} drts_problem;

/* Batched step (n_rhs > 1) implementations (Eq. 26 with R right-hand sides
 * sharing A; both within 1e-5 of the FP64 oracle over 1500 steps):
 *   DRTS_BATCHED_CUDA_CORES  sliced sparse A, one pass per tile of 4..32 rhs,
 *                            compensated FP32 sums; state kept in groups of
 *                            four right-hand sides;
 *   DRTS_BATCHED_TENSOR      tcgen05 tensor cores, all rhs in one pass
 *                            (DRTS_FP32 precision, n_rhs <= 64): A stored per
 *                            voxel and neighbour role at the problem's union
 *                            of block positions, as three bf16 terms (the
 *                            first an integer of <= 9 bits times a
 *                            power-of-two row scale, so each tile's leading
 *                            products sum exactly), the state as three bf16
 *                            terms per value, FP32 sums per output; the
 *                            faster form. */
#define DRTS_BATCHED_CUDA_CORES 0
#define DRTS_BATCHED_TENSOR 1

typedef struct drts_ctx drts_ctx;

/* Sizes of an assembled context (bytes are device bytes). */
typedef struct drts_info {
    int64_t n_states;                /* 26 * nx*ny*nz */
    int64_t nnz;                     /* stored nonzeros of A (no padding) */
    int64_t nnz_padded;              /* slots in the sliced format incl. padding */
    int64_t n_slices;                /* slices of 32 rows */
    int64_t matrix_bytes;            /* values + codes + row scales + slice table */
    int64_t state_bytes;             /* one state buffer, all right-hand sides */
    int64_t t;                       /* steps taken so far */
    int32_t precision, n_rhs, n_patch;
    int32_t special_voxels_permille; /* voxels that needed edge/interface folding */
    int64_t nnz_stored;              /* entries the step streams (no padding): nnz, plus
                                        for DRTS_FP16_ROWSCALE the second FP16 term of
                                        each large value stored as two (hi + lo) */
} drts_info;

/*
 * Assemble the system matrix A of Eq. 23 on the device (Eq. 18-21 with the
 * Section 4.2 edge and interface treatment) and allocate the state, the
 * detector history and the energy ledger for n_rhs right-hand sides.
 * The state starts at zero and t at 0.  cuda_stream is a cudaStream_t (or
 * NULL).  On success *out owns everything; on failure *out is NULL.
 */
drts_status drts_assemble(const drts_problem *prob, void *cuda_stream, drts_ctx **out);

/*
 * Set the source term of right-hand side rhs (Eq. 26, B P(t)):
 *   s(t) = sum_e weight[e] * P(t) * e_{state_idx[e]},
 *   P(t) = profile[t - t0] for t0 <= t < t0 + n_t, else 0.
 * state_idx are canonical state indices (host int64), weight and profile are
 * host FP64; 0 <= n_entries <= 64, 0 <= n_t.  Replaces any earlier source of
 * that rhs.  The term lands in x(t+1) when stepping from t.
 */
drts_status drts_inject_source(drts_ctx *ctx, int32_t rhs, int32_t n_entries,
                               const int64_t *state_idx, const double *weight,
                               int64_t t0, int32_t n_t, const double *profile);

/*
 * Advance every right-hand side by n_steps (Fig. 3 loop): for each step,
 * x(t+1) = A x(t) + s(t), and from x(t) the detector readout
 * det[t][p] = sum over states s of patch p of exit_det(s) x(t)[s] (Eq. 27)
 * plus the FP64 absorbed / exited ledger.  Asynchronous on the context
 * stream.  DRTS_EINVAL if t + n_steps exceeds max_steps.
 */
drts_status drts_step_n(drts_ctx *ctx, int64_t n_steps);

/*
 * Copy the detector history of rhs for steps [t_begin, t_end) to host_out
 * ([t][patch], FP64, caller-owned, (t_end-t_begin)*n_patch values) and, if
 * ledger_out is not NULL, the ledger {sum of x(t), injected, absorbed,
 * exited} (4 FP64, cumulative since t = 0).  Synchronises the stream.
 * DRTS_EINVAL for a bad rhs or a range outside [0, t]; DRTS_ESTATE for a
 * non-empty range without a detector history (det_face none or max_steps 0).
 */
drts_status drts_read_detectors(drts_ctx *ctx, int32_t rhs, int64_t t_begin,
                                int64_t t_end, double *host_out, double *ledger_out);

/*
 * Point detectors: Eq. 27 with a general sparse F (Section 4.2 places a
 * sensor anywhere in the volume; a point detector reads chosen
 * (voxel, direction) states).  Detector d of rhs r reads, at every step t,
 *   pdet[r][t][d] = sum over entries e with det[e] = d of weight[e] * x_t[state_idx[e]]
 * from x(t), the state the step starts from (the face detector's timing).
 * n_entries (state, detector, weight) triples, host arrays, copied; entries of
 * one detector are summed in their given order with a fixed reduction (the
 * readout is deterministic).  0 <= n_det <= 65535; n_det = 0 removes them;
 * a new set replaces (and frees) the previous one, a rejected call keeps it.
 * The history holds max_steps steps (DRTS_ESTATE when max_steps is 0) and
 * is cleared by this call; steps before it read 0.  While point detectors
 * are set, t + n_steps may not exceed max_steps.  Works in every step mode
 * and for every right-hand side.  Synchronises.
 */
drts_status drts_set_point_detectors(drts_ctx *ctx, int32_t n_det, int64_t n_entries,
                                     const int32_t *det, const int64_t *state_idx,
                                     const double *weight);

/* Copy the point-detector history of rhs for steps [t_begin, t_end) to
 * host_out ([t][n_det] FP64, caller-owned).  Synchronises.  DRTS_ESTATE if
 * no point detectors are set. */
drts_status drts_read_point_detectors(drts_ctx *ctx, int32_t rhs, int64_t t_begin,
                                      int64_t t_end, double *host_out);

/*
 * Sensor response of Eq. 27: a sensor integrates the photons it receives
 * with an impulse response h over a window of +-w steps,
 *   M[t][d] = sum over k in [t - w, t + w], 0 <= k < t_rec, of h[t - k + w] D[k][d],
 * where D is the recorded readout of rhs (which = DRTS_SENSOR_FACE: the face
 * patches, DRTS_SENSOR_POINT: the point detectors), h[j + w] the response at
 * lag j steps (2w+1 host FP64 taps, 0 <= w <= 2^20) and t_rec = min(t,
 * max_steps) the steps recorded so far.  Writes M for t in [t_begin, t_end)
 * (t_end <= t_rec) to host_out ([t][d] FP64).  Products and sums are rounded
 * separately in k order.  Synchronises.
 */
#define DRTS_SENSOR_FACE 0
#define DRTS_SENSOR_POINT 1
drts_status drts_sensor_response(drts_ctx *ctx, int32_t rhs, int32_t which, int64_t t_begin,
                                 int64_t t_end, int32_t w, const double *h, double *host_out);

/*
 * Source partition within a step (Section 4.1: for accuracy the source
 * function is sampled in time intervals of dr/c, shorter than the step).
 *
 * drts_source_column: where a unit population is at the end of a step when
 * it leaves the centre of voxel i in direction n (state_idx = i*26 + n) and
 * travels only the fraction frac (0 < frac <= 1) of the step's path L_k:
 * Eq. 18/19/21 evaluated for the path frac * L_k, folded at the domain edge
 * and at interfaces as the first-order system matrix is.  frac = 1 is
 * column state_idx of A under DRTS_INTERFACE_FIRST_ORDER (under TWO_STEP
 * the columns of crossing states differ); as frac -> 0 the population stays
 * in state_idx.  Writes the target
 * states (ascending) and values to host arrays of capacity cap; *count
 * receives the number of targets (DRTS_EINVAL, with *count set, if it
 * exceeds cap) and, if exit_mass is not NULL, *exit_mass the mass that
 * leaves the grid.  FP64.  Synchronises.
 *
 * drts_inject_source_substeps: sub-step source of right-hand side rhs.
 * Entry e (state_idx[e], weight[e]) emits weight[e] * profile[(t - t0) *
 * n_sub + j] in sub-interval j of step t (0 <= j < n_sub, t0 <= t < t0 +
 * n_t).  Sub-interval j is taken at its midpoint, so its population travels
 * frac_j = 1 - (j + 1/2) / n_sub of the step and lands in x(t+1) as
 * drts_source_column(state_idx[e], frac_j).  1 <= n_sub <= 64; the
 * paper's dr/c partition is drts_substep_count's n_sub.  0 <= n_entries <=
 * 64; n_entries = 0 removes rhs's sub-step source.
 * Replaces any earlier sub-step source of rhs and adds to the plain source
 * of drts_inject_source.  The ledger's injected mass counts what lands in
 * the state.  Not available in the persistent step mode nor with
 * drts_run_host (DRTS_EUNSUPPORTED).  Synchronises.
 */
/* drts_substep_count: the number of sub-intervals of length dr/c in one step
 * of the medium of state_idx's voxel: its path L_k in half voxels (2 dr =
 * h), rounded up (2 when L_k = h). */
drts_status drts_substep_count(drts_ctx *ctx, int64_t state_idx, int32_t *n_sub);
drts_status drts_source_column(drts_ctx *ctx, int64_t state_idx, double frac, int32_t cap,
                               int64_t *out_state, double *out_value, int32_t *count,
                               double *exit_mass);
drts_status drts_inject_source_substeps(drts_ctx *ctx, int32_t rhs, int32_t n_entries,
                                        const int64_t *state_idx, const double *weight,
                                        int32_t n_sub, int64_t t0, int32_t n_t,
                                        const double *profile);

/* Copy x(t) of rhs to host_out (canonical order, n_states FP64, caller-owned).
 * Synchronises.  DRTS_EINVAL for a bad rhs or a NULL buffer. */
drts_status drts_read_state(drts_ctx *ctx, int32_t rhs, double *host_out);

/* Overwrite x(t) of rhs from host_in (canonical order, n_states FP64,
 * caller-owned, read during the call, rounded to the state precision).  t is
 * unchanged.  Synchronises.  DRTS_EINVAL for a bad rhs or a NULL buffer. */
drts_status drts_write_state(drts_ctx *ctx, int32_t rhs, const double *host_in);

/*
 * End-to-end run from host memory: for each of n_steps steps, copy that
 * step's source scale factors host->device (scale[i*n_rhs + r] multiplies the
 * injected weights of rhs r at step t+i, replacing P(t)), advance one step,
 * and copy that step's detector readout device->host into
 * det_out[i][r][patch] (NULL: no readout).  Both buffers are caller-owned;
 * pinned host memory lets the copies overlap.  Synchronises at the end.
 * DRTS_EINVAL for a NULL scale or as drts_step_n; DRTS_EUNSUPPORTED while
 * sub-step sources are set.
 */
drts_status drts_run_host(drts_ctx *ctx, int64_t n_steps, const double *scale,
                          double *det_out);

/*
 * Export rows [row_begin, row_end) of the assembled A in canonical CSR form
 * (rows in canonical state order, columns ascending): row_ptr has
 * row_end-row_begin+1 entries starting at 0, col and val have room for cap
 * entries (DRTS_EINVAL if too small; row_ptr is still filled).  Values are
 * the stored ones (FP64, FP32, or FP16 times the row scale) widened to FP64;
 * a value kept as two FP16 terms is exported as their sum, so the structure
 * is the matrix's in every precision.  Synchronises.
 */
drts_status drts_export_rows(drts_ctx *ctx, int64_t row_begin, int64_t row_end,
                             int64_t *row_ptr, int32_t *col, double *val, int64_t cap);

/* Per-state column functionals of the step (canonical order, n_states FP64
 * each, any may be NULL): absorbed fraction 1-exp(-mu_a L) (Eq. 8), fraction
 * leaving the grid, fraction leaving through the detector face (Eq. 27). */
drts_status drts_column_info(drts_ctx *ctx, double *absorb, double *exit_total,
                             double *exit_det);

/* Sizes and step count of ctx (drts_info above) into *out.  Does not
 * synchronise.  DRTS_EINVAL for a NULL argument. */
drts_status drts_get_info(const drts_ctx *ctx, drts_info *out);

/*
 * Host-built tables of one medium of a problem, computed without a device
 * (a diagnostic of the inputs the device assembler reads; the step does not
 * need it).  Outputs are caller-owned FP64/FP32 arrays, any may be NULL:
 *   stencil_out    [26][27][26]: W_k[n][o][m], the mass a state of direction
 *                  n in a voxel of medium k sends in one step to the voxel at
 *                  offset o (index (oz+1)*9 + (oy+1)*3 + (ox+1)) in direction
 *                  m (Eq. 18, 19, 21), before edge or interface folding;
 *   exit_total_out [27][26]: fraction of a state of medium k, direction n,
 *                  that leaves the grid in one step, by the voxel's face mask
 *                  bz*9 + by*3 + bx (b = 0 at the low face, 1 inside, 2 at
 *                  the high face of that axis; Section 4.2 with R4);
 *   exit_det_out   [27][26]: the part of it that leaves through the detector
 *                  face (Eq. 27);
 *   dir_scale_out  [26]: the FP16 tier's power-of-two row scale per direction
 *                  (1 for the other precisions).
 * DRTS_EINVAL for a problem drts_assemble would reject or a medium outside
 * 0..n_media-1 (message in drts_last_error(NULL)).
 */
drts_status drts_host_tables(const drts_problem *prob, int32_t medium, double *stencil_out,
                             double *exit_total_out, double *exit_det_out, float *dir_scale_out);

/*
 * Host-built two-step entries of a DRTS_INTERFACE_TWO_STEP problem (Section
 * 4.2, planar interface crossed in two parts), computed without a device: a
 * state in a voxel of medium k1 whose z neighbour layer holds medium k2.
 * Outputs are caller-owned, any may be NULL:
 *   cross_out [26]: 1 when direction n reaches the plane between the layers
 *                   within the step (those states use the entries below
 *                   instead of medium k1's stencil), else 0;
 *   fold_out  [26][27][26]: mass scattered before the plane, by target
 *                   offset o and direction m (folded at edges and interfaces
 *                   as the stencil is);
 *   edge_out  [26][27][26]: mass reflected or refracted at the plane (folded
 *                   at the grid edge only).
 * DRTS_EINVAL for a problem drts_assemble would reject, interface !=
 * DRTS_INTERFACE_TWO_STEP, or media k1, k2 that do not meet across a z plane
 * with different refractive indices.
 */
drts_status drts_two_step_tables(const drts_problem *prob, int32_t k1, int32_t k2, uint8_t *cross_out,
                                 double *fold_out, double *edge_out);

/* Set the launch shape of the step kernel (0 = library default): blocks per
 * SM (must fit), threads per block (multiple of 32, <= 256), right-hand sides
 * per pass of the batched step, and the kernel variant (-1 keeps the current
 * one; 0-2 = matrix streamed into registers with 1-3 groups prefetched, 3-6 =
 * matrix streamed into shared-memory stages by bulk async copies, stage
 * shapes (groups, stages) = (8,3), (4,3), (4,4), (2,6); 7-8 = state halo of
 * each 32-voxel block staged in shared memory, 13 or 26 warps, grids with nx
 * a multiple of 32 only; 9 = registers path with the matrix stream two groups
 * ahead and the x gathers of the next group in flight; 10-11 = two or four
 * warps per slice, each summing a contiguous part of the rows, for grids too
 * small to give every warp slot a slice; 12-13 = registers path with one
 * group in flight and 32-bit slice, voxel and state indices, compiled for six
 * or eight 256-thread blocks per SM; 14 = eight warps per slice, blocks of
 * 256 threads).  For a batched
 * context on the CUDA cores the variant is the slice order: 0 = warps
 * stride over all slices, 1 = block-major (one CTA works through all 26
 * direction slices of a voxel block), 2 = block-major with the block's x
 * halo staged in shared memory (fixed shape: 26 warps, one CTA per SM, 4
 * FP32 / 2 FP64 right-hand sides per pass; rhs_tile, threads and blocks are
 * ignored); the tensor-core form has variant 0 only.  All variants compute the same step; they differ only in speed.
 * DRTS_EINVAL if the shape does not fit on an SM or the variant is unknown. */
drts_status drts_set_launch(drts_ctx *ctx, int32_t blocks_per_sm,
                            int32_t threads_per_block, int32_t rhs_tile,
                            int32_t variant);

/*
 * How drts_step_n issues its steps (Fig. 3 loop):
 *   DRTS_STEP_LAUNCH      one kernel launch per step (default);
 *   DRTS_STEP_PERSISTENT  one cooperative launch runs all n steps, with a
 *                         grid-wide barrier between steps whose wait is
 *                         bounded (DRTS_ETIMEOUT instead of a hang); for
 *                         small grids where launch gaps matter.  One
 *                         right-hand side only.
 * DRTS_EINVAL for an unknown mode; DRTS_EUNSUPPORTED for the persistent mode
 * with several right-hand sides, with sub-step sources set, or where the
 * device offers no cooperative launch.  Takes effect at the next step.
 */
#define DRTS_STEP_LAUNCH 0
#define DRTS_STEP_PERSISTENT 1
drts_status drts_set_step_mode(drts_ctx *ctx, int32_t mode);

/*
 * Checkpoint / resume.  A checkpoint holds t, the state of every right-hand
 * side (canonical order, FP64), the ledger and the face- and point-detector
 * histories up to t; A itself is not stored (it is rebuilt by drts_assemble
 * from the same problem, deterministically) and neither are the sources and
 * point-detector definitions (set them again before loading).
 * drts_checkpoint_size gives the bytes needed, drts_checkpoint_save writes
 * them into a caller-owned host buffer, and drts_checkpoint_load restores
 * them into a context assembled from the same problem with the same number
 * of point detectors (DRTS_EINVAL otherwise).  Stepping on from a restored
 * context gives the same states as the uninterrupted run.  Synchronous.
 */
drts_status drts_checkpoint_size(drts_ctx *ctx, int64_t *bytes);
drts_status drts_checkpoint_save(drts_ctx *ctx, void *host_buf, int64_t cap);
drts_status drts_checkpoint_load(drts_ctx *ctx, const void *host_buf, int64_t size);

/* Result of drts_autotune. */
typedef struct drts_tune_result {
    int32_t variant, threads, blocks_per_sm, rhs_tile;
    double ms_per_step;              /* measured time of the chosen launch */
    int32_t candidates;              /* launches timed (0 when from the cache) */
    int32_t from_cache;
} drts_tune_result;

/*
 * Pick the fastest launch of the step for this context by timing every
 * variant, block size and blocks-per-SM choice that fits (trial_steps timed
 * launches each, CUDA events on the context stream; the four fastest are then
 * timed twice more, alternately, over 3 x trial_steps launches, and the best
 * of those repeats wins) and apply it.  The state,
 * t, detectors and ledger are left unchanged (the trial steps write the spare
 * state buffer and a scratch ledger).  Results are cached per (grid,
 * precision, rhs, SM count, stored entries) in the process and, when the environment
 * variable DRTS_TUNE_CACHE names a file, appended to it and read back by later
 * processes.  Synchronises.  out may be NULL.
 */
drts_status drts_autotune(drts_ctx *ctx, int32_t trial_steps, drts_tune_result *out);

/*
 * Host-side fault injection for testing the failure paths (no GPU fault is
 * ever caused).  kind:
 *   DRTS_FAULT_NONE        clear everything below;
 *   DRTS_FAULT_SKIP_COPY   the bulk-copy step variants (3-6, one right-hand
 *                          side; DRTS_ESTATE for any other launch) never issue
 *                          copy number arg of the first warp, so that warp's
 *                          bounded wait runs out; the step then reports
 *                          DRTS_ETIMEOUT at the next synchronising call and the
 *                          context stays usable;
 *   DRTS_FAULT_SPIN_LIMIT  polls before a device-side wait gives up (arg,
 *                          1..2^30; default 2^22);
 *   DRTS_FAULT_SKIP_BARRIER in persistent mode the first block never arrives
 *                          at the first grid barrier, so the other blocks'
 *                          bounded waits run out (DRTS_ETIMEOUT).
 */
#define DRTS_FAULT_NONE 0
#define DRTS_FAULT_SKIP_COPY 1
#define DRTS_FAULT_SPIN_LIMIT 2
#define DRTS_FAULT_SKIP_BARRIER 3   /* persistent mode: the first block never
                                       arrives at the first grid barrier */
drts_status drts_set_fault(drts_ctx *ctx, int32_t kind, int64_t arg);

/* Device allocator for the buffers of contexts made by drts_assemble
 * (process-wide, all threads; read at each allocation).  alloc_fn(bytes,
 * cuda_stream, user) returns device memory of at least `bytes` bytes aligned
 * to 256 bytes, or NULL when it has none (the call that needed it then
 * fails with DRTS_ENOMEM); free_fn(ptr, cuda_stream, user) takes it back
 * after the context's stream has drained.  A buffer is freed with the
 * functions that allocated it, so the allocator may change while contexts
 * live.  Both NULL restores cudaMalloc / cudaFree; one NULL is DRTS_EINVAL.
 * This lets a framework's caching allocator (PyTorch's) own the library's
 * device memory.  Temporary buffers of single calls and the close-packed
 * contexts keep the stream-ordered CUDA allocator. */
typedef void *(*drts_alloc_fn)(size_t bytes, void *cuda_stream, void *user);
typedef void (*drts_free_fn)(void *ptr, void *cuda_stream, void *user);
drts_status drts_set_allocator(drts_alloc_fn alloc_fn, drts_free_fn free_fn, void *user);

/* Host-side allocator fault for tests (process-wide, all threads): after
 * `n_ok` further device allocations of context buffers succeed, the next one
 * fails as if the device were out of memory, without calling the allocator;
 * later ones succeed again.  The failing call returns DRTS_ENOMEM and frees
 * what it allocated (drts_assemble frees the partial context and sets *out
 * to NULL).  A negative n_ok disarms the fault.  Always DRTS_OK. */
drts_status drts_set_alloc_fault(int64_t n_ok);

/*
 * Sum of x(t) of right-hand side rhs (the "sum of x" term of the ledger that
 * drts_read_detectors returns), written to out_device: one FP64 value in
 * device memory the caller owns.  The paper has no counterpart to this call.
 * drts_read_detectors allocates a small device buffer for the same sum; this
 * call allocates nothing, for callers that cannot allocate device memory when
 * they need the sum: real-time loops that must not wait on the allocator's
 * locks or latency, and processes whose device memory is owned and budgeted
 * by another runtime's pool.  Its per-block partial sums live in a static
 * device array of 4096 doubles (32 KiB) that every GPU which loads the
 * library keeps until the process exits.
 *   - Limit: at most 268,435,456 states (4096 blocks of 65,536); larger state
 *     vectors are rejected with DRTS_EINVAL.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it for the life of the process; make
 *     that first call before any stream capture.  A device reset
 *     (cudaDeviceReset) invalidates the cached address: do not call this
 *     entry point on a device after resetting it.
 *   - Every call shares the array.  Calls on one stream are ordered; calls
 *     whose kernels overlap on the GPU (other streams, other contexts on the
 *     same device) race on it and may return wrong sums.
 *   - Asynchronous on the context stream; the result is deterministic (fixed
 *     reduction order) and equals the ledger's sum up to rounding order.
 *   - DRTS_EUNSUPPORTED for a context of the tensor-core batched step
 *     (batched_kernel DRTS_BATCHED_TENSOR with n_rhs > 1), whose state
 *     layout this reduction does not read.
 */
drts_status drts_state_sum_noalloc(drts_ctx *ctx, int32_t rhs, double *out_device);

/* ------------------------------------------------------------------------
 * Serving loop: continuous batching of independent simulations.
 *
 * The paper's method assembles A once per medium and then only steps it
 * (Fig. 3); a server keeps many such simulations resident at once.  Requests
 * queue on the host.  Each drts_server_tick (1) captures the next
 * steps_per_tick steps of every resident simulation into one CUDA graph whose
 * branches fan out over n_streams streams (their kernels overlap on the
 * device) and launches it, (2) while it runs, admits queued requests in
 * the configured order as long as a resident slot and device memory (a footprint
 * estimate against mem_budget_bytes) are free, assembling their A, and (3)
 * retires finished simulations: detector history and ledger are copied to
 * host and their device memory is freed.  A request submitted while others
 * run is admitted at a later tick.  Results do not depend on what else is
 * resident (each simulation's kernels read only its own data).
 * ------------------------------------------------------------------------ */
typedef struct drts_server drts_server;

/* Admission order of queued requests: DRTS_SERVE_FIFO admits in arrival
 * order; DRTS_SERVE_SHORTEST_FIRST admits the queued request with the least
 * estimated work (voxels x 26 x passes over A per step x steps) first, which
 * lowers the median latency of a burst; under sustained overload it can keep
 * postponing large requests (there is no ageing). */
#define DRTS_SERVE_FIFO 0
#define DRTS_SERVE_SHORTEST_FIRST 1

typedef struct drts_server_config {
    int64_t mem_budget_bytes;        /* device bytes for resident simulations; 0 = 90% of free */
    int32_t max_resident;            /* resident simulations at once, 1..256 */
    int32_t steps_per_tick;          /* steps each resident simulation advances per tick */
    int32_t n_streams;               /* streams a tick's graph fans out over, 1..32 */
    int32_t policy;                  /* DRTS_SERVE_FIFO or DRTS_SERVE_SHORTEST_FIRST */
    int32_t keep_state;              /* nonzero: keep each finished request's final state
                                        x(n_steps) of every rhs on the host (FP64, canonical
                                        order) for drts_server_result_state */
    int32_t reserved;                /* must be 0 */
} drts_server_config;

#define DRTS_REQ_QUEUED 0
#define DRTS_REQ_RUNNING 1
#define DRTS_REQ_DONE 2
#define DRTS_REQ_FAILED 3
#define DRTS_REQ_CANCELLED 4

typedef struct drts_request_info {
    int32_t state;                   /* DRTS_REQ_* */
    int32_t n_rhs, n_patch;
    int64_t n_steps;
    int64_t footprint_bytes;         /* device bytes reserved while resident */
    double queue_s;                  /* submit -> admission (host clock) */
    double latency_s;                /* submit -> completion (host clock) */
} drts_request_info;

/* Counters since creation; resident, queued and used_bytes are the counts at
 * the time of the call. */
typedef struct drts_server_stats {
    int64_t submitted, admitted, completed, failed, ticks, graph_launches;
    int32_t resident, queued;
    int64_t used_bytes, budget_bytes;
    /* the tick graph: ticks whose executable graph was updated in place
     * (same launches, new parameters), ticks that instantiated a new one,
     * host seconds spent capturing and updating / instantiating in all
     * ticks, and the part of it in the ticks that instantiated */
    int64_t graph_updates, graph_instantiations;
    double host_graph_s, host_instantiate_s;
    int64_t cancelled;               /* requests withdrawn by drts_server_cancel */
} drts_server_stats;

/* Create a server on the current device (cfg is copied; *out owns its
 * streams and every request).  DRTS_EINVAL for a configuration out of range,
 * DRTS_ECUDA if the device or its streams cannot be set up. */
drts_status drts_server_create(const drts_server_config *cfg, drts_server **out);

/* Queue one simulation: problem (copied; max_steps is set to n_steps), its
 * sources as n_entries (rhs, canonical state, weight) triples sharing one
 * time profile P(t0 .. t0+n_t-1) (Eq. 26), and the number of steps.  Returns
 * at once with the request id.  DRTS_ENOMEM if the request could never fit
 * the budget. */
drts_status drts_server_submit(drts_server *srv, const drts_problem *prob, int32_t n_entries,
                               const int32_t *src_rhs, const int64_t *src_state,
                               const double *src_weight, int64_t t0, int32_t n_t,
                               const double *profile, int64_t n_steps, int64_t *request_id);

/* One scheduling round (see above); *n_done = simulations retired.  A
 * request whose assembly or result readout fails is marked DRTS_REQ_FAILED
 * (drts_server_result then reports its error) and the others go on. */
drts_status drts_server_tick(drts_server *srv, int32_t *n_done);

/* State, sizes and host-clock timings of a request.  DRTS_EINVAL for an
 * unknown id. */
drts_status drts_server_poll(drts_server *srv, int64_t request_id, drts_request_info *out);

/* Detector history [n_steps][n_patch] and ledger {sum x, injected, absorbed,
 * exited} of right-hand side rhs of a finished request (caller-owned host
 * buffers, either may be NULL).  DRTS_ESTATE before the request is done,
 * DRTS_EINVAL for an unknown id or rhs. */
drts_status drts_server_result(drts_server *srv, int64_t request_id, int32_t rhs,
                               double *det_out, double *ledger_out);
/* Final state x(n_steps) of right-hand side rhs of a finished request
 * (n_states FP64 values in canonical order into caller-owned state_out),
 * kept only when the server was created with keep_state set.  DRTS_ESTATE
 * before the request is done or when states are not kept, DRTS_EINVAL for an
 * unknown id, rhs or a NULL buffer. */
drts_status drts_server_result_state(drts_server *srv, int64_t request_id, int32_t rhs,
                                     double *state_out);
/* Withdraw a queued or running request.  A queued one leaves the queue; a
 * running one is stopped between ticks: the call waits for the server's
 * streams (nothing of the simulation is then in flight), frees its device
 * memory and returns its footprint to the budget.  The request ends in
 * DRTS_REQ_CANCELLED with no results (drts_server_result reports
 * DRTS_ESTATE) until it is released.  DRTS_ESTATE for a request that has
 * already finished, failed or been cancelled, DRTS_EINVAL for an unknown id,
 * DRTS_ECUDA if waiting for the device fails. */
drts_status drts_server_cancel(drts_server *srv, int64_t request_id);
/* Forget a finished, failed or cancelled request and its results
 * (DRTS_ESTATE while it is queued or running, DRTS_EINVAL for an unknown
 * id). */
drts_status drts_server_release(drts_server *srv, int64_t request_id);
drts_status drts_server_get_stats(const drts_server *srv, drts_server_stats *out);
/* Text of the server's last error ("" for NULL); valid until the next call. */
const char *drts_server_last_error(const drts_server *srv);
/* Wait for the device, free every request and the server (NULL is ignored). */
void drts_server_destroy(drts_server *srv);

/* Free every device and host resource of ctx (NULL is ignored). */
void drts_destroy(drts_ctx *ctx);

/* Text of the last error on ctx (or, when ctx is NULL, of the last failed
 * drts_assemble on the calling thread).  Valid until the next call on ctx
 * (or the thread's next drts_assemble). */
const char *drts_last_error(const drts_ctx *ctx);

/* ---- Close-packed sphere partition (Section 3) ------------------------
 *
 * The paper partitions the medium into touching spheres of radius dr in
 * close packing (face-centred cubic).  Sites: integer triples (i, j, k) with
 * i + j + k even, 0 <= i < nx (nx even), 0 <= j < ny, 0 <= k < nz, centred
 * at (i, j, k) * 2dr / sqrt(2); site index ((k*ny + j)*nx + i) / 2.
 * Directions: the 12 unit vectors towards the nearest neighbours,
 * (dx, dy, dz) / sqrt(2) with two nonzero components, dz slowest and dx
 * fastest; state index site*12 + d.  One step moves light 2dr (all media
 * share one refractive index: there is no interface folding), and the edges
 * are open: mass whose target site lies outside the box leaves.  The matrix
 * follows Eq. 18-21 and 23 as on the voxel grid.  drts_fcc_host_rows is the
 * host assembly (FP64 rows); drts_fcc_assemble and the calls after it run the
 * step on the device.
 */
typedef struct drts_fcc_problem {
    int32_t nx, ny, nz;              /* integer box; nx even, ny, nz >= 1 */
    double spacing_mm;               /* 2dr, the distance of touching sphere centres */
    int32_t n_media;                 /* 1..255, one refractive index */
    const drts_medium *media;        /* [n_media], host, read during the call */
    const uint8_t *medium_of_site;   /* [nx*ny*nz/2] in site order, host */
} drts_fcc_problem;

/*
 * Rows [row_begin, row_end) of the close-packed partition's matrix A,
 * assembled on the host in FP64: row_ptr [row_end - row_begin + 1] relative
 * to row_begin, col / val [cap] with ascending columns per row (caller-owned).
 * DRTS_EINVAL for a bad problem, row range or a cap below the entry count
 * (row_ptr is filled either way); messages in drts_last_error(NULL).
 */
drts_status drts_fcc_host_rows(const drts_fcc_problem *prob, int64_t row_begin, int64_t row_end,
                               int64_t *row_ptr, int32_t *col, double *val, int64_t cap);

/*
 * ---- The step on the close-packed partition, on the device ----
 *
 * The same Eq. 26 step x(t+1) = A x(t) + s(t) (x(0) = 0) on the close-packed
 * sites, with A of Eq. 18-21 and 23 assembled on the device: the host builds
 * only each medium's FP64 stencil (transition weights by lattice offset and
 * direction pair); device kernels count, lay out (SELL-32 slices of 32
 * consecutive sites of one direction, 16-bit codes offset*12 + n) and fill
 * the rows, each row's entries in ascending column order.  Values and state
 * in FP64 (DRTS_FP64) or FP32 (DRTS_FP32).  All calls are on the stream given
 * to drts_fcc_assemble; those that return host data synchronise it.
 */
typedef struct drts_fcc_ctx drts_fcc_ctx;

typedef struct drts_fcc_info {
    int64_t n_sites;
    int64_t n_states;                /* n_sites * 12 */
    int64_t nnz;                     /* stored nonzeros */
    int64_t slots;                   /* entries including slice padding */
    int32_t n_offsets;               /* lattice offsets of the stencil (the site itself included) */
    int32_t precision;
    int64_t t;                       /* steps taken */
    int64_t matrix_bytes;            /* values + codes on the device */
} drts_fcc_info;

/*
 * Validates prob (as drts_fcc_host_rows), assembles A on the device and
 * returns a context with x = 0, t = 0.  precision: DRTS_FP64 or DRTS_FP32
 * (DRTS_EUNSUPPORTED otherwise).  cuda_stream: a cudaStream_t or NULL for the
 * default stream.  Host inputs are read during the call only.  DRTS_EINVAL /
 * DRTS_ENOMEM / DRTS_ECUDA with a message in drts_last_error(NULL).
 */
drts_status drts_fcc_assemble(const drts_fcc_problem *prob, int32_t precision, void *cuda_stream,
                              drts_fcc_ctx **out);

/*
 * The source term s(t) of Eq. 26: s(t) = P(t) sum_e weights[e] e_{states[e]}
 * with P(t) = profile[t - t0] for t0 <= t < t0 + n_t, else 0 (t counts the
 * steps taken; step t adds s(t)).  states index n_sites * 12 (site * 12 + d),
 * at most 64 entries; the arrays are copied.  Replaces an earlier source.
 */
drts_status drts_fcc_set_source(drts_fcc_ctx *ctx, int32_t n, const int64_t *states, const double *weights,
                                int64_t t0, int32_t n_t, const double *profile);

/* n steps of Eq. 26 on the context's stream (asynchronous). */
drts_status drts_fcc_step_n(drts_fcc_ctx *ctx, int64_t n);

/* x(t) in state order (site * 12 + d) as FP64, host_out [n_states], caller-owned. */
drts_status drts_fcc_read_state(drts_fcc_ctx *ctx, double *host_out);

/*
 * Rows [row_begin, row_end) (state order) of the assembled A read back from
 * the device as CSR: row_ptr [row_end - row_begin + 1] relative to
 * row_begin, col / val [cap] (caller-owned; val in FP64 whatever the stored
 * precision).  DRTS_EINVAL for a bad range or a cap below the entry count
 * (row_ptr is filled either way).
 */
drts_status drts_fcc_read_rows(drts_fcc_ctx *ctx, int64_t row_begin, int64_t row_end, int64_t *row_ptr,
                               int32_t *col, double *val, int64_t cap);

drts_status drts_fcc_get_info(const drts_fcc_ctx *ctx, drts_fcc_info *out);

/* Frees the context (NULL is a no-op); the stream is drained first. */
drts_status drts_fcc_destroy(drts_fcc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DRTS_H */
