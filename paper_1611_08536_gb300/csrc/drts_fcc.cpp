// Host assembly of the DRTS matrix on the close-packed sphere partition of
// Section 3 of arXiv:1611.08536 (face-centred cubic packing of equal spheres
// of radius dr).
//
// Sites are integer triples (i, j, k) with an even coordinate sum, in units
// of a = 2dr / sqrt(2), so touching spheres are s = sqrt(2) a apart; the 12
// directions point at the nearest neighbours.  One step moves light L = s
// (one refractive index for all media).  For a source state (site, n) the
// unscattered share is spread around B = L S_n (Eq. 18) and the scattered
// share over the segment A_m B for every m (Eq. 19), both over the sites
// strictly closer than s, weights (s - d) / sum; contributions to one target
// state add (Eq. 20-21).  Targets outside the box leave (open edges).
//
// Rows are gathered: row (site j, direction m) collects, for each stencil
// offset o with a transition into m, the source site j - o and every source
// direction n, in ascending source-state order.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "drts_internal.h"

namespace drts {
namespace {

struct Vec3 {
    double x, y, z;
};

Vec3 operator-(Vec3 a, Vec3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
Vec3 operator+(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
Vec3 operator*(double t, Vec3 a) { return {t * a.x, t * a.y, t * a.z}; }
double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// nearest-neighbour offsets (two nonzero components), dz slowest, dx fastest
struct FccDirs {
    int v[kFccDirs][3];
    Vec3 u[kFccDirs];
    FccDirs()
    {
        int d = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if ((dx != 0) + (dy != 0) + (dz != 0) != 2) continue;
                    v[d][0] = dx; v[d][1] = dy; v[d][2] = dz;
                    const double r = 1.0 / std::sqrt(2.0);
                    u[d] = {dx * r, dy * r, dz * r};
                    ++d;
                }
    }
};

const FccDirs &fcc_dirs()
{
    static const FccDirs D;
    return D;
}

double seg_dist(Vec3 p, Vec3 a, Vec3 b)
{
    const Vec3 d = b - a;
    const double dd = dot(d, d);
    if (dd == 0.0) return std::sqrt(dot(p - b, p - b));
    double t = dot(p - a, d) / dd;
    t = std::min(1.0, std::max(0.0, t));
    const Vec3 q = a + t * d;
    return std::sqrt(dot(p - q, p - q));
}

// Transitions of one medium: for every offset of the stencil (lattice
// offsets that receive anything), W[o][n][m].
struct FccStencil {
    std::vector<std::array<int, 3>> off;
    std::vector<double> W;                 // [off][12][12]
    double &at(size_t o, int n, int m) { return W[(o * kFccDirs + n) * kFccDirs + m]; }
    double at(size_t o, int n, int m) const { return W[(o * kFccDirs + n) * kFccDirs + m]; }
};

FccStencil fcc_stencil(const drts_medium &med, double spacing_mm)
{
    const FccDirs &D = fcc_dirs();
    const double s = std::sqrt(2.0);       // neighbour distance in units of a
    const double L = s;                    // one refractive index: L = s
    const double p_un = std::exp(-med.mu_s * spacing_mm) * std::exp(-med.mu_a * spacing_mm);
    const double p_sc = (1.0 - std::exp(-med.mu_s * spacing_mm)) * std::exp(-med.mu_a * spacing_mm);
    // discrete Henyey-Greenstein table, rows normalised
    double G[kFccDirs][kFccDirs];
    for (int n = 0; n < kFccDirs; ++n) {
        double tot = 0.0;
        for (int m = 0; m < kFccDirs; ++m) {
            const double mu = dot(D.u[n], D.u[m]);
            G[n][m] = (1.0 - med.g * med.g) / std::pow(1.0 + med.g * med.g - 2.0 * med.g * mu, 1.5);
            tot += G[n][m];
        }
        for (int m = 0; m < kFccDirs; ++m) G[n][m] /= tot;
    }
    // candidate lattice offsets: even coordinate sum, within L + s
    std::vector<std::array<int, 3>> cand;
    for (int z = -3; z <= 3; ++z)
        for (int y = -3; y <= 3; ++y)
            for (int x = -3; x <= 3; ++x)
                if (((x + y + z) & 1) == 0 && std::sqrt(double(x * x + y * y + z * z)) < L + s + 1e-9)
                    cand.push_back({x, y, z});
    std::vector<double> acc(cand.size() * kFccDirs * kFccDirs, 0.0);
    std::vector<double> w(cand.size());
    // spread share over the candidates strictly closer than s (the distance
    // of each from the point or segment in dist[]), weights (s - d) / sum
    auto spread = [&](const std::vector<double> &dist, int n, int m, double share) {
        double tot = 0.0;
        for (size_t c = 0; c < cand.size(); ++c) {
            w[c] = dist[c] * dist[c] < s * s * (1.0 - 1e-9) ? s - dist[c] : 0.0;
            tot += w[c];
        }
        if (tot <= 0.0) return;
        for (size_t c = 0; c < cand.size(); ++c)
            if (w[c] > 0.0) acc[(c * kFccDirs + n) * kFccDirs + m] += share * (w[c] / tot);
    };
    std::vector<double> dist(cand.size());
    for (int n = 0; n < kFccDirs; ++n) {
        const Vec3 B = L * D.u[n];
        if (p_un > 0.0) {                                     // Eq. 18
            for (size_t c = 0; c < cand.size(); ++c) {
                const Vec3 X{double(cand[c][0]), double(cand[c][1]), double(cand[c][2])};
                dist[c] = std::sqrt(dot(X - B, X - B));
            }
            spread(dist, n, n, p_un);
        }
        if (p_sc > 0.0) {                                     // Eq. 19
            for (int m = 0; m < kFccDirs; ++m) {
                const Vec3 A = L * D.u[m];
                for (size_t c = 0; c < cand.size(); ++c) {
                    const Vec3 X{double(cand[c][0]), double(cand[c][1]), double(cand[c][2])};
                    dist[c] = seg_dist(X, A, B);
                }
                spread(dist, n, m, G[n][m] * p_sc);
            }
        }
    }
    FccStencil S;
    for (size_t c = 0; c < cand.size(); ++c) {
        bool any = false;
        for (int q = 0; q < kFccDirs * kFccDirs && !any; ++q) any = acc[c * kFccDirs * kFccDirs + q] > 0.0;
        if (!any) continue;
        S.off.push_back(cand[c]);
        S.W.insert(S.W.end(), acc.begin() + c * kFccDirs * kFccDirs, acc.begin() + (c + 1) * kFccDirs * kFccDirs);
    }
    return S;
}

drts_status fcc_fail(const std::string &m)
{
    set_global_error(m);
    return DRTS_EINVAL;
}

}  // namespace

drts_status fcc_validate(const drts_fcc_problem *p)
{
    if (!p) return fcc_fail("problem is NULL");
    if (p->nx < 2 || p->ny < 1 || p->nz < 1 || (p->nx & 1)) return fcc_fail("nx must be even and >= 2, ny, nz >= 1");
    if (!(p->spacing_mm > 0.0)) return fcc_fail("spacing_mm must be > 0");
    if (p->n_media < 1 || p->n_media > 255 || !p->media || !p->medium_of_site)
        return fcc_fail("n_media must be 1..255 with media and medium_of_site");
    const int64_t n_sites = int64_t(p->nx) * p->ny * p->nz / 2;
    if (n_sites * kFccDirs >= (int64_t(1) << 31)) return fcc_fail("more than 2^31 states");
    for (int k = 0; k < p->n_media; ++k) {
        const drts_medium &m = p->media[k];
        if (!(m.n > 0.0) || m.mu_s < 0.0 || m.mu_a < 0.0 || !(m.g > -1.0 && m.g < 1.0))
            return fcc_fail("medium " + std::to_string(k) + " out of range");
        if (m.n != p->media[0].n) return fcc_fail("all media need one refractive index (no interface folding)");
    }
    for (int64_t v = 0; v < n_sites; ++v)
        if (p->medium_of_site[v] >= p->n_media) return fcc_fail("medium index out of range");
    return DRTS_OK;
}

// The stencils of all media on one list of lattice offsets (the union of
// the offsets any medium reaches, plus the site itself, which the device
// step uses for padding entries): W[k][o][n][m].
void fcc_tables(const drts_fcc_problem &p, FccTables &T)
{
    std::vector<FccStencil> S;
    for (int k = 0; k < p.n_media; ++k) S.push_back(fcc_stencil(p.media[k], p.spacing_mm));
    T.off.clear();
    T.off.push_back({0, 0, 0});
    for (const FccStencil &Sk : S)
        for (const auto &o : Sk.off)
            if (std::find(T.off.begin(), T.off.end(), o) == T.off.end()) T.off.push_back(o);
    const size_t no = T.off.size();
    T.W.assign(size_t(p.n_media) * no * kFccDirs * kFccDirs, 0.0);
    for (int k = 0; k < p.n_media; ++k)
        for (size_t o = 0; o < S[size_t(k)].off.size(); ++o) {
            const size_t u = size_t(std::find(T.off.begin(), T.off.end(), S[size_t(k)].off[o]) - T.off.begin());
            for (int n = 0; n < kFccDirs; ++n)
                for (int m = 0; m < kFccDirs; ++m)
                    T.W[((size_t(k) * no + u) * kFccDirs + n) * kFccDirs + m] = S[size_t(k)].at(o, n, m);
        }
}

}  // namespace drts

using namespace drts;

extern "C" {

drts_status drts_fcc_host_rows(const drts_fcc_problem *p, int64_t row_begin, int64_t row_end,
                               int64_t *row_ptr, int32_t *col, double *val, int64_t cap)
try {
    const drts_status st = fcc_validate(p);
    if (st != DRTS_OK) return st;
    const int64_t n_states = int64_t(p->nx) * p->ny * p->nz / 2 * kFccDirs;
    if (row_begin < 0 || row_end < row_begin || row_end > n_states || !row_ptr) return fcc_fail("bad row range");

    std::vector<FccStencil> S;
    for (int k = 0; k < p->n_media; ++k) S.push_back(fcc_stencil(p->media[k], p->spacing_mm));
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    std::vector<std::pair<int64_t, double>> row;
    row_ptr[0] = 0;
    int64_t out = 0;
    for (int64_t r = row_begin; r < row_end; ++r) {
        const int64_t j = r / kFccDirs;
        const int m = int(r % kFccDirs);
        // site j is the h-th of its lattice row (jj, kk), which holds the
        // nx / 2 sites i = 2h + ((jj + kk) & 1)
        const int64_t rowi = j / (nx / 2);
        const int h = int(j - rowi * (nx / 2));
        const int jj = int(rowi % ny), kk = int(rowi / ny);
        const int ii = 2 * h + ((jj + kk) & 1);
        row.clear();
        // the offsets differ between media only in their values, so take
        // each medium's stencil as it is and read the source's medium
        for (int k = 0; k < p->n_media; ++k) {
            const FccStencil &Sk = S[size_t(k)];
            for (size_t o = 0; o < Sk.off.size(); ++o) {
                const int si = ii - Sk.off[o][0], sj = jj - Sk.off[o][1], sk = kk - Sk.off[o][2];
                if (si < 0 || si >= nx || sj < 0 || sj >= ny || sk < 0 || sk >= nz) continue;
                const int64_t src = ((int64_t(sk) * ny + sj) * nx + si) / 2;
                if (p->medium_of_site[src] != k) continue;
                for (int n = 0; n < kFccDirs; ++n) {
                    const double w = Sk.at(o, n, m);
                    if (w > 0.0) row.emplace_back(src * kFccDirs + n, w);
                }
            }
        }
        std::sort(row.begin(), row.end());
        for (const auto &e : row) {
            if (out < cap && col && val) {
                col[out] = int32_t(e.first);
                val[out] = e.second;
            }
            ++out;
        }
        row_ptr[r - row_begin + 1] = out;
    }
    if (out > cap || (out > 0 && (!col || !val)))
        return fcc_fail("capacity " + std::to_string(cap) + " < " + std::to_string(out) + " entries");
    return DRTS_OK;
} catch (const std::bad_alloc &) {
    set_global_error("drts_fcc_host_rows: host allocation failed");
    return DRTS_ENOMEM;
} catch (...) {
    set_global_error("drts_fcc_host_rows: unexpected exception");
    return DRTS_EINVAL;
}

}  // extern "C"
