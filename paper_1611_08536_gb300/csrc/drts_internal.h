// Internal declarations shared by the library's translation units.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "drts.h"

namespace drts {

// Named NVTX range over a scope: assembly, steps, autotuning, checkpoints and
// serving ticks appear by name in profiler timelines and can select ncu
// captures (nothing is recorded unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kDirs = 26;         // lattice directions
constexpr int kOffs = 27;         // neighbour offsets {-1,0,1}^3
constexpr int kCodes = kOffs * kDirs;  // column code = offset_index*26 + direction
constexpr int kSlice = 32;        // rows per slice (one warp, one lane per row)
constexpr int kGroup = 4;         // entries per lane per vector load
constexpr int kCenterCode = 13 * kDirs;  // offset (0,0,0), direction 0: padding
constexpr int kMaxRhs = 64;
constexpr int kMaxSrc = 64;

// Close-packed (FCC) partition: 12 nearest-neighbour directions.
constexpr int kFccDirs = 12;

// Stencils of every medium of a close-packed problem on one list of lattice
// offsets (offset 0 is the site itself): W[k][o][n][m], FP64, host-built.
struct FccTables {
    std::vector<std::array<int, 3>> off;
    std::vector<double> W;
};
drts_status fcc_validate(const drts_fcc_problem *p);   // DRTS_EINVAL with a message
void fcc_tables(const drts_fcc_problem &p, FccTables &T);

// Lattice direction table (state order of Eq. 22).
struct Directions {
    int v[kDirs][3];      // integer vector
    double u[kDirs][3];   // unit vector S_d
    int nnzc[kDirs];      // number of nonzero components (1 axis, 2 edge, 3 corner)
    int index_of[27];     // (dz+1)*9+(dy+1)*3+(dx+1) -> direction (-1 at origin)
    Directions();
};
const Directions &dirs();

#ifdef __CUDACC__
#define DRTS_HD __host__ __device__
#else
#define DRTS_HD
#endif

DRTS_HD inline int offset_index(int dx, int dy, int dz) { return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1); }

// Host-built tables of one problem (FP64).  Transcendentals (exp, sqrt, the
// Henyey-Greenstein power, Fresnel) are evaluated here once; the device
// assembler only looks them up and multiplies.
struct HostTables {
    int n_media = 0;
    std::vector<double> lam;        // [k] L_k / h
    std::vector<double> nref;       // [k] refractive index
    std::vector<double> absorb;     // [k] 1 - exp(-mu_a L_k)
    // raw stencil W[k][n][o][m]: mass sent from direction n of a voxel of
    // medium k to the voxel at offset o in direction m (Eq. 18, 19, 21)
    std::vector<double> W;          // [k][26][27][26]
    // plain-row templates: for row direction m and column offset index d
    // (source = row voxel + d), the entries (n, W[k][n][26-d][m]) with W > 0
    std::vector<int32_t> tmpl_off;  // [k][26][28]
    std::vector<uint8_t> tmpl_n;
    std::vector<double> tmpl_val;
    // Fresnel reflectance by incidence class c (0: cos 0, else 1/sqrt(c)
    // with c nonzero direction components): edge [k][4], interface [k1][k2][4]
    std::vector<double> r_edge;     // [k][4]
    std::vector<double> r_int;      // [k][k][4]
    // exit fractions of a state of medium k in a voxel whose face mask is
    // mask = bz*9+by*3+bx (b = 0 low face, 1 inside, 2 high face)
    std::vector<double> exit_total; // [k][27][26]
    std::vector<double> exit_det;   // [k][27][26]
    std::vector<float> dir_scale;   // [26] FP16 tier: row scale of direction m (power of two)
    int n_template_entries_max = 0;

    // Planar two-step interface crossing (DRTS_INTERFACE_TWO_STEP, Section
    // 4.2): the ordered medium pairs (k1 of a source voxel, k2 of the z layer
    // next to it) with different refractive indices that meet in the grid,
    // and for each pair the raw entries of every direction that reaches the
    // plane between them within the step.
    int n_pairs = 0;
    std::vector<int32_t> pair_slot; // [K][K] slot of (k1, k2), or -1
    std::vector<uint8_t> cross;     // [P][26] 1: direction n reaches the plane within the step
    std::vector<double> W2f;        // [P][26][27][26] raw entries folded at edges and interfaces
    std::vector<double> W2n;        // [P][26][27][26] raw entries folded at the grid edge only

    // Ledger classes of the column functionals (absorbed and exiting mass of
    // a state in one step): class = medium, or with two-step interfaces one
    // class per distinct (medium, pair above, pair below) of a z layer.
    int n_classes = 0;
    std::vector<uint8_t> class_of_layer;  // [nz] (two-step interfaces only; else class = medium)
    std::vector<double> led_absorb;       // [C] absorbed fraction of a non-crossing state
    std::vector<double> led_absorb_dir;   // [C][26] per direction (two-step interfaces only)
    std::vector<double> led_exit_total;   // [C][27][26] as exit_total, per class
    std::vector<double> led_exit_det;     // [C][27][26] as exit_det, per class
};

// path_frac scales every medium's path L_k (1 for the system matrix; a
// fraction of the step for sources emitted within it, Section 4.1)
std::string build_host_tables(const drts_problem &p, HostTables &t, double path_frac = 1.0);
// the two-step interface part of build_host_tables (problem already validated
// to one medium per z layer); fills pair_slot .. W2n and the ledger classes
std::string build_two_step_tables(const drts_problem &p, HostTables &t);

// Record the message drts_last_error(NULL) returns on this thread (calls
// that have no context).
void set_global_error(const std::string &msg);

}  // namespace drts
