// Host-side FP64 tables of the DRTS system matrix (Section 3 and 4.2 of
// arXiv:1611.08536).  Everything here runs once per problem; the per-row work
// of assembling A happens in the device assembler (drts_assemble.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include <cuda_fp16.h>

#include "drts_internal.h"

namespace drts {

Directions::Directions()
{
    int d = 0;
    for (int &x : index_of) x = -1;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                v[d][0] = dx; v[d][1] = dy; v[d][2] = dz;
                double len = std::sqrt(double(dx * dx + dy * dy + dz * dz));
                u[d][0] = dx / len; u[d][1] = dy / len; u[d][2] = dz / len;
                nnzc[d] = (dx != 0) + (dy != 0) + (dz != 0);
                index_of[offset_index(dx, dy, dz)] = d;
                ++d;
            }
}

const Directions &dirs()
{
    static const Directions D;
    return D;
}

namespace {

// Squared distance from the lattice point p (units of h) to the closed
// segment from a to b; a == b degenerates to the point distance.
double dist2_to_segment(const double p[3], const double a[3], const double b[3])
{
    double e[3], w[3];
    for (int c = 0; c < 3; ++c) { e[c] = b[c] - a[c]; w[c] = p[c] - a[c]; }
    double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    double s = 0.0;
    if (ee > 0.0) {
        s = (w[0] * e[0] + w[1] * e[1] + w[2] * e[2]) / ee;
        s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
    }
    double r = 0.0;
    for (int c = 0; c < 3; ++c) {
        double q = w[c] - s * e[c];
        r += q * q;
    }
    return r;
}

// Unpolarised Fresnel reflectance at incidence cosine ci from index n1 into
// n2; 1 under total internal reflection, 0 when the indices match.
double fresnel(double ci, double n1, double n2)
{
    if (n1 == n2) return 0.0;
    double st = n1 / n2 * std::sqrt(1.0 - ci * ci);
    if (st >= 1.0) return 1.0;
    double ct = std::sqrt(1.0 - st * st);
    double a = (n1 * ci - n2 * ct) / (n1 * ci + n2 * ct);
    double b = (n1 * ct - n2 * ci) / (n1 * ct + n2 * ci);
    return 0.5 * (a * a + b * b);
}

// Nearest-neighbour weights of Eq. 18/19 around the segment [a, b] (a point
// when a == b): (1 - dist)/sum over offsets strictly closer than 2dr = h.
// Points exactly one voxel away are excluded whatever the rounding: the
// squared distance must be below 1 - 1e-9.
void segment_weights(const double a[3], const double b[3], double wout[kOffs])
{
    double sum = 0.0;
    for (int o = 0; o < kOffs; ++o) {
        double p[3] = {double(o % 3 - 1), double(o / 3 % 3 - 1), double(o / 9 - 1)};
        double d2 = dist2_to_segment(p, a, b);
        wout[o] = d2 < 1.0 - 1e-9 ? 1.0 - std::sqrt(d2) : 0.0;
        sum += wout[o];
    }
    for (int o = 0; o < kOffs; ++o) wout[o] /= sum;
}

// Error-diffused rounding of one medium's stencil to FP32.  Each source
// direction n owns a column of A (its ~210 targets (o, m)); plain rounding
// to nearest leaves every column sum off by a small amount that is the same
// for all interior columns of that direction, so the total mass drifts by
// about 1e-8 per step.  Rounding the entries largest first, each to the
// neighbouring float that keeps the running sum of rounding errors nearest
// zero, makes the FP32 column sum match the FP64 one to the last entry's
// rounding.  Every entry is one of the two floats bracketing its FP64 value.
void diffuse_round_fp32(const double *W, double *out)
{
    std::vector<int> idx;
    for (int n = 0; n < kDirs; ++n) {
        idx.clear();
        for (int o = 0; o < kOffs; ++o)
            for (int m = 0; m < kDirs; ++m)
                if (W[(n * kOffs + o) * kDirs + m] > 0.0) idx.push_back(o * kDirs + m);
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
            return W[n * kOffs * kDirs + a] > W[n * kOffs * kDirs + b];
        });
        double resid = 0.0;
        for (int e : idx) {
            const double v = W[n * kOffs * kDirs + e];
            // the two floats bracketing v (equal when v is a float)
            const float f = float(v);
            float lo = f, hi = f;
            if (double(f) > v) lo = std::nextafter(f, 0.0f);
            else if (double(f) < v) hi = std::nextafter(f, 2.0f);
            const double a = double(lo), b = double(hi);
            const double pick = std::fabs(resid + a - v) <= std::fabs(resid + b - v) ? a : b;
            out[n * kOffs * kDirs + e] = pick;
            resid += pick - v;
        }
    }
}

// Mass of one raw column Wn[o][m] (a state of a medium with edge
// reflectances r_edge[4], in a voxel with face mask `mask`) that leaves the
// grid in one step, and the part of it through the detector face: a raw
// target outside the grid along axis a (x, then y, then z) keeps R and lets
// 1 - R out through that face (Section 4.2 edge reading).
void column_exit(const double *Wn, const double *r_edge, int mask, int det_face, double &tot, double &det)
{
    const Directions &D = dirs();
    const int b[3] = {mask % 3, mask / 3 % 3, mask / 9};
    tot = 0.0;
    det = 0.0;
    for (int o = 0; o < kOffs; ++o) {
        const int ov[3] = {o % 3 - 1, o / 3 % 3 - 1, o / 9 - 1};
        for (int m = 0; m < kDirs; ++m) {
            double w = Wn[o * kDirs + m];
            if (w <= 0.0) continue;
            for (int a = 0; a < 3; ++a) {
                const bool out_lo = b[a] == 0 && ov[a] == -1;
                const bool out_hi = b[a] == 2 && ov[a] == 1;
                if (!out_lo && !out_hi) continue;
                const int c = D.v[m][a] != 0 ? D.nnzc[m] : 0;
                const double R = r_edge[c];
                const double leave = w * (1.0 - R);
                tot += leave;
                if (det_face == 2 * a + (out_hi ? 1 : 0)) det += leave;
                w *= R;
            }
        }
    }
}

// Share of the sphere of lattice direction m in the discrete kernel
// (DRTS_HG_QUADRATURE): the weights of the degree-7 rule on the 26
// directions, fixed by the octahedral moments 1, x^4, x^2 y^2 and x^2 y^2 z^2
// (sphere averages 1, 1/5, 1/15, 1/105): 6 a + 12 b + 8 c = 1,
// 2 a + 2 b + 8 c / 9 = 1/5, b + 8 c / 9 = 1/15, 8 c / 27 = 1/105, so
// a = 1/21 (axes), b = 4/105 (face diagonals), c = 9/280 (body diagonals).
double direction_share(int mode, int m)
{
    if (mode != DRTS_HG_QUADRATURE) return 1.0;
    switch (dirs().nnzc[m]) {
    case 1: return 1.0 / 21.0;
    case 2: return 4.0 / 105.0;
    default: return 9.0 / 280.0;
    }
}

// Henyey-Greenstein weights of the 26 lattice directions for scattering out
// of the unit vector u, normalised over the lattice (the discrete kernel of
// Section 5, here also for a direction that is not a lattice one); with
// DRTS_HG_QUADRATURE each direction also carries its share of the sphere.
void phase_row(double g, int mode, const double u[3], double out[kDirs])
{
    const Directions &D = dirs();
    double sum = 0.0;
    for (int m = 0; m < kDirs; ++m) {
        const double mu = u[0] * D.u[m][0] + u[1] * D.u[m][1] + u[2] * D.u[m][2];
        const double den = 1.0 + g * g - 2.0 * g * mu;
        out[m] = (1.0 - g * g) / (den * std::sqrt(den));
        if (mode == DRTS_HG_QUADRATURE) out[m] *= direction_share(mode, m);
        sum += out[m];
    }
    for (int m = 0; m < kDirs; ++m) out[m] /= sum;
}

// Mass w landing around the segment [a, b] (points in units of h, a point
// when a == b) in direction m, shared over the lattice offsets by the
// weights of Eq. 18/19, added to the raw column Wn[o][m].
void deposit(double *Wn, const double a[3], const double b[3], int m, double w)
{
    if (!(w > 0.0)) return;
    double wo[kOffs];
    segment_weights(a, b, wo);
    for (int o = 0; o < kOffs; ++o)
        if (wo[o] > 0.0) Wn[o * kDirs + m] += wo[o] * w;
}

// One free flight (Eq. 9-12 and 18/19 for a population that starts at the
// point c instead of a voxel centre): mass `mass` leaves c along the unit
// vector u for the path l (units of h) in medium md.  The unscattered share
// lands around c + l u, divided over the lattice states st[0..ns) by the
// shares sh; the scattered share lands around [c + l S_m, c + l u] in every
// direction m, weighted by the phase row ph.
void flight(double *Wn, const double c[3], const double u[3], double l, double h, const drts_medium &md,
            const double ph[kDirs], const int *st, const double *sh, int ns, double mass)
{
    const Directions &D = dirs();
    const double end[3] = {c[0] + l * u[0], c[1] + l * u[1], c[2] + l * u[2]};
    const double keep = mass * std::exp(-(md.mu_s + md.mu_a) * l * h);
    for (int q = 0; q < ns; ++q) deposit(Wn, end, end, st[q], keep * sh[q]);
    const double scat = mass * (1.0 - std::exp(-md.mu_s * l * h)) * std::exp(-md.mu_a * l * h);
    if (scat > 0.0)
        for (int m = 0; m < kDirs; ++m) {
            const double a[3] = {c[0] + l * D.u[m][0], c[1] + l * D.u[m][1], c[2] + l * D.u[m][2]};
            deposit(Wn, a, end, m, scat * ph[m]);
        }
}

// Raw column of a state of direction n in a voxel of medium k1 whose z
// neighbour layer holds medium k2 (another refractive index), when S_n
// reaches the plane between them, half a voxel away, within the step
// (Section 4.2, planar interface crossed in two parts).  With lambda_1 the
// path of a whole step in medium 1 (units of h), the plane is met at the
// fraction tc = 1/2 / (lambda_1 |S_nz|) of the step; tc >= 1 returns false
// (no crossing).  Writes
//  * Wf: the share scattered before the plane.  A photon scattered at the
//    fraction s < tc into m ends the step at lambda_1 (s S_n + (1 - s) S_m):
//    a segment from lambda_1 S_m to lambda_1 (tc S_n + (1 - tc) S_m), with
//    the scattering probability of the path tc L_1 and the absorption of the
//    whole step in medium 1.  These entries meet the interface again in the
//    assembler's fold.
//  * Wn: the unscattered share exp(-(mu_s1 + mu_a1) tc L_1) at the crossing
//    point C = tc lambda_1 S_n.  The Fresnel share R at the true incidence
//    angle continues in medium 1 along S_n with z reversed; the rest is
//    refracted by Snell's law (sin t = n1/n2 sin i, same azimuth) and
//    continues in medium 2 for (1 - tc) of a step at medium 2's speed.  The
//    refracted direction is not a lattice direction: its population goes to
//    the two lattice directions of its azimuth whose polar angles bracket
//    its own (the normal and S_n, or S_n and the horizontal), linearly in the
//    polar angle.  These entries meet no further interface in the step.
// Snell's law cannot give total reflection here: tc < 1 needs lambda_1 |S_nz|
// > 1/2, so n1 < 2 n_min |S_nz| <= 2 n2 |S_nz|, and sin t = n1/n2 sin i < 1
// follows from 4 cos^2 i sin^2 i <= 1.
bool two_step_column(const drts_problem &p, double nmin, int k1, int k2, int n, double *Wf, double *Wn)
{
    const Directions &D = dirs();
    if (D.v[n][2] == 0) return false;
    const drts_medium &m1 = p.media[k1], &m2 = p.media[k2];
    const double lam1 = nmin / m1.n, lam2 = nmin / m2.n;
    const double ci = std::fabs(D.u[n][2]);            // cosine of incidence on the plane
    const double tc = 0.5 / (lam1 * ci);
    if (!(tc < 1.0)) return false;
    const double h = p.voxel_mm;
    const double zs = D.v[n][2] > 0 ? 1.0 : -1.0;

    // scattered before the plane
    double ph1[kDirs];
    phase_row(m1.g, p.direction_weights, D.u[n], ph1);
    const double p_scat = (1.0 - std::exp(-m1.mu_s * tc * lam1 * h)) * std::exp(-m1.mu_a * lam1 * h);
    if (p_scat > 0.0)
        for (int m = 0; m < kDirs; ++m) {
            const double a[3] = {lam1 * D.u[m][0], lam1 * D.u[m][1], lam1 * D.u[m][2]};
            double b[3];
            for (int c = 0; c < 3; ++c) b[c] = lam1 * (tc * D.u[n][c] + (1.0 - tc) * D.u[m][c]);
            deposit(Wf, a, b, m, p_scat * ph1[m]);
        }

    // unscattered up to the crossing point, then reflected and refracted
    const double p_keep = std::exp(-(m1.mu_s + m1.mu_a) * tc * lam1 * h);
    const double C[3] = {tc * lam1 * D.u[n][0], tc * lam1 * D.u[n][1], tc * lam1 * D.u[n][2]};
    const double R = fresnel(ci, m1.n, m2.n);
    const int nr = D.index_of[offset_index(D.v[n][0], D.v[n][1], -D.v[n][2])];
    double phr[kDirs];
    phase_row(m1.g, p.direction_weights, D.u[nr], phr);
    const double one = 1.0;
    flight(Wn, C, D.u[nr], (1.0 - tc) * lam1, h, m1, phr, &nr, &one, 1, p_keep * R);
    if (R < 1.0) {
        const double si = std::sqrt(1.0 - ci * ci);
        const double st = m1.n / m2.n * si;
        const double ct = std::sqrt(1.0 - st * st);
        double u[3] = {0.0, 0.0, zs * ct};
        int states[2] = {n, n};
        double share[2] = {1.0, 0.0};
        int ns = 1;
        if (si > 0.0) {
            const double hor = std::sqrt(D.u[n][0] * D.u[n][0] + D.u[n][1] * D.u[n][1]);
            u[0] = st * D.u[n][0] / hor;
            u[1] = st * D.u[n][1] / hor;
            const double th_i = std::atan2(si, ci), th_t = std::atan2(st, ct);
            const double right = 1.57079632679489661923;   // pi / 2
            if (th_t <= th_i) {            // between the normal and S_n
                states[1] = D.index_of[offset_index(0, 0, D.v[n][2])];
                share[0] = th_t / th_i;
            } else {                       // between S_n and the horizontal
                states[1] = D.index_of[offset_index(D.v[n][0], D.v[n][1], 0)];
                share[0] = (right - th_t) / (right - th_i);
            }
            share[1] = 1.0 - share[0];
            ns = 2;
        }
        double ph2[kDirs];
        phase_row(m2.g, p.direction_weights, u, ph2);
        flight(Wn, C, u, (1.0 - tc) * lam2, h, m2, ph2, states, share, ns, p_keep * (1.0 - R));
    }
    return true;
}

}  // namespace

// Two-step tables of every medium pair that meets across a z plane, and the
// ledger classes of the layers (problems validated to one medium per layer).
std::string build_two_step_tables(const drts_problem &p, HostTables &t)
{
    const int K = p.n_media;
    const int64_t layer = int64_t(p.nx) * p.ny;
    double nmin = p.media[0].n;
    for (int k = 1; k < K; ++k) nmin = std::fmin(nmin, p.media[k].n);
    std::vector<int> kz(size_t(p.nz));
    for (int z = 0; z < p.nz; ++z) kz[size_t(z)] = p.medium_of_voxel[int64_t(z) * layer];

    const size_t blk = size_t(kDirs) * kOffs * kDirs;
    t.pair_slot.assign(size_t(K) * K, -1);
    t.n_pairs = 0;
    std::vector<std::pair<int, int>> pairs;
    for (int z = 0; z + 1 < p.nz; ++z) {
        const int a = kz[size_t(z)], b = kz[size_t(z) + 1];
        if (p.media[a].n == p.media[b].n) continue;
        for (const auto &pr : {std::make_pair(a, b), std::make_pair(b, a)})
            if (t.pair_slot[size_t(pr.first) * K + pr.second] < 0) {
                t.pair_slot[size_t(pr.first) * K + pr.second] = int32_t(pairs.size());
                pairs.push_back(pr);
            }
    }
    t.n_pairs = int(pairs.size());
    t.cross.assign(size_t(t.n_pairs) * kDirs, 0);
    t.W2f.assign(size_t(t.n_pairs) * blk, 0.0);
    t.W2n.assign(size_t(t.n_pairs) * blk, 0.0);
    for (int q = 0; q < t.n_pairs; ++q)
        for (int n = 0; n < kDirs; ++n) {
            const size_t off = size_t(q) * blk + size_t(n) * kOffs * kDirs;
            t.cross[size_t(q) * kDirs + n] =
                two_step_column(p, nmin, pairs[size_t(q)].first, pairs[size_t(q)].second, n, &t.W2f[off],
                                &t.W2n[off]);
        }

    // ledger classes: (medium, slot of the pair above, slot of the pair below)
    std::vector<std::array<int, 3>> keys;
    t.class_of_layer.assign(size_t(p.nz), 0);
    for (int z = 0; z < p.nz; ++z) {
        const int k = kz[size_t(z)];
        const int up = z + 1 < p.nz ? t.pair_slot[size_t(k) * K + kz[size_t(z) + 1]] : -1;
        const int dn = z > 0 ? t.pair_slot[size_t(k) * K + kz[size_t(z) - 1]] : -1;
        const std::array<int, 3> key = {k, up, dn};
        size_t c = 0;
        while (c < keys.size() && keys[c] != key) ++c;
        if (c == keys.size()) {
            if (keys.size() == 255)
                return "two-step interfaces: more than 255 distinct (medium, neighbour layers) classes";
            keys.push_back(key);
        }
        t.class_of_layer[size_t(z)] = uint8_t(c);
    }
    const int C = int(keys.size());
    t.n_classes = C;
    t.led_absorb.assign(size_t(C), 0.0);
    t.led_absorb_dir.assign(size_t(C) * kDirs, 0.0);
    t.led_exit_total.assign(size_t(C) * 27 * kDirs, 0.0);
    t.led_exit_det.assign(size_t(C) * 27 * kDirs, 0.0);
    std::vector<double> col(size_t(kOffs) * kDirs);
    for (int c = 0; c < C; ++c) {
        const int k = keys[size_t(c)][0];
        t.led_absorb[size_t(c)] = t.absorb[size_t(k)];
        for (int n = 0; n < kDirs; ++n) {
            const Directions &D = dirs();
            const int slot = D.v[n][2] > 0 ? keys[size_t(c)][1] : (D.v[n][2] < 0 ? keys[size_t(c)][2] : -1);
            const bool crossing = slot >= 0 && t.cross[size_t(slot) * kDirs + n];
            double kept = 0.0;
            if (crossing) {
                const size_t off = size_t(slot) * blk + size_t(n) * kOffs * kDirs;
                for (size_t e = 0; e < col.size(); ++e) {
                    col[e] = t.W2f[off + e] + t.W2n[off + e];
                    kept += col[e];
                }
            } else {
                std::copy_n(&t.W[size_t(k) * blk + size_t(n) * kOffs * kDirs], col.size(), col.begin());
            }
            // a crossing state keeps what its raw entries carry; the rest is absorbed
            t.led_absorb_dir[size_t(c) * kDirs + n] = crossing ? 1.0 - kept : t.absorb[size_t(k)];
            for (int mask = 0; mask < 27; ++mask) {
                const size_t ti = (size_t(c) * 27 + mask) * kDirs + n;
                column_exit(col.data(), &t.r_edge[size_t(k) * 4], mask, p.det_face, t.led_exit_total[ti],
                            t.led_exit_det[ti]);
            }
        }
    }
    return std::string();
}

std::string build_host_tables(const drts_problem &p, HostTables &t, double path_frac)
{
    const Directions &D = dirs();
    const int K = p.n_media;
    t.n_media = K;
    double nmin = p.media[0].n;
    for (int k = 1; k < K; ++k) nmin = std::fmin(nmin, p.media[k].n);

    t.lam.assign(K, 0.0);
    t.nref.assign(K, 0.0);
    t.absorb.assign(K, 0.0);
    t.W.assign(size_t(K) * kDirs * kOffs * kDirs, 0.0);
    for (int k = 0; k < K; ++k) {
        const drts_medium &md = p.media[k];
        const double lam = path_frac * nmin / md.n;   // path / h  (L_k = h n_min / n_k)
        const double L = lam * p.voxel_mm;
        const double keep_a = std::exp(-md.mu_a * L);      // Eq. 8
        const double keep_s = std::exp(-md.mu_s * L);      // Eq. 3 / 6
        const double unscat = keep_s * keep_a;             // Eq. 9
        const double scat = (1.0 - keep_s) * keep_a;       // Eq. 10
        t.lam[k] = lam;
        t.nref[k] = md.n;
        t.absorb[k] = 1.0 - keep_a;
        double *Wk = &t.W[size_t(k) * kDirs * kOffs * kDirs];
        for (int n = 0; n < kDirs; ++n) {
            // discrete Henyey-Greenstein kernel from S_n, normalised over m
            // (each m weighted by its share of the sphere with DRTS_HG_QUADRATURE)
            double phase[kDirs], psum = 0.0;
            for (int m = 0; m < kDirs; ++m) {
                double mu = D.u[n][0] * D.u[m][0] + D.u[n][1] * D.u[m][1] + D.u[n][2] * D.u[m][2];
                double den = 1.0 + md.g * md.g - 2.0 * md.g * mu;
                phase[m] = (1.0 - md.g * md.g) / (den * std::sqrt(den));
                if (p.direction_weights == DRTS_HG_QUADRATURE) phase[m] *= direction_share(p.direction_weights, m);
                psum += phase[m];
            }
            const double B[3] = {lam * D.u[n][0], lam * D.u[n][1], lam * D.u[n][2]};
            double w[kOffs];
            if (unscat > 0.0) {                            // Eq. 11 and 18
                segment_weights(B, B, w);
                for (int o = 0; o < kOffs; ++o)
                    Wk[(n * kOffs + o) * kDirs + n] += w[o] * unscat;
            }
            if (scat > 0.0) {                              // Eq. 12 and 19
                for (int m = 0; m < kDirs; ++m) {
                    const double A[3] = {lam * D.u[m][0], lam * D.u[m][1], lam * D.u[m][2]};
                    segment_weights(A, B, w);
                    const double f = phase[m] / psum * scat;
                    for (int o = 0; o < kOffs; ++o)
                        Wk[(n * kOffs + o) * kDirs + m] += w[o] * f;   // Eq. 21
                }
            }
        }
    }

    // stencil values as stored by the plain rows: FP64 as computed, FP32 with
    // column-preserving rounding, FP16 as computed (rounded at fill time)
    std::vector<double> Wstore(t.W);
    if (p.precision == DRTS_FP32)
        for (int k = 0; k < K; ++k) {
            const size_t off = size_t(k) * kDirs * kOffs * kDirs;
            diffuse_round_fp32(&t.W[off], &Wstore[off]);
        }
    // FP16 tier: every row of direction m is stored as FP16 times a power of
    // two scale[m] chosen so the largest value of any medium maps to 2^14
    // (the FP16 normal range then covers values down to ~4e-9 of it)
    t.dir_scale.assign(kDirs, 1.0f);
    if (p.precision == DRTS_FP16_ROWSCALE) {
        for (int m = 0; m < kDirs; ++m) {
            double mx = 0.0;
            for (int k = 0; k < K; ++k)
                for (int n = 0; n < kDirs; ++n)
                    for (int o = 0; o < kOffs; ++o)
                        mx = std::fmax(mx, t.W[((size_t(k) * kDirs + n) * kOffs + o) * kDirs + m]);
            const int e2 = mx > 0.0 ? int(std::ceil(std::log2(mx))) : 0;
            t.dir_scale[m] = std::ldexp(1.0f, e2 - 14);
        }
        // the FP16 values are rounded per entry in the fill kernel (spatially
        // dithered), so the templates keep the FP64 values
    }

    // plain-row templates (row direction m, column offset d = source - row)
    t.tmpl_off.assign(size_t(K) * kDirs * (kOffs + 1), 0);
    t.tmpl_n.clear();
    t.tmpl_val.clear();
    t.n_template_entries_max = 0;
    for (int k = 0; k < K; ++k) {
        const double *Wk = &Wstore[size_t(k) * kDirs * kOffs * kDirs];
        for (int m = 0; m < kDirs; ++m) {
            int32_t *off = &t.tmpl_off[(size_t(k) * kDirs + m) * (kOffs + 1)];
            int row_entries = 0;
            for (int d = 0; d < kOffs; ++d) {
                off[d] = int32_t(t.tmpl_n.size());
                const int o = kOffs - 1 - d;   // target offset seen from the source
                for (int n = 0; n < kDirs; ++n) {
                    double v = Wk[(n * kOffs + o) * kDirs + m];
                    if (v > 0.0) {
                        t.tmpl_n.push_back(uint8_t(n));
                        t.tmpl_val.push_back(v);
                        ++row_entries;
                    }
                }
            }
            off[kOffs] = int32_t(t.tmpl_n.size());
            if (row_entries > t.n_template_entries_max) t.n_template_entries_max = row_entries;
        }
    }

    // Fresnel classes: 0 grazing (cos 0), c = 1, 2, 3 nonzero components
    auto class_cos = [](int c) { return c == 0 ? 0.0 : 1.0 / std::sqrt(double(c)); };
    t.r_edge.assign(size_t(K) * 4, 0.0);
    t.r_int.assign(size_t(K) * K * 4, 0.0);
    for (int k = 0; k < K; ++k)
        for (int c = 0; c < 4; ++c) {
            double R = p.boundary == DRTS_MIRROR ? 1.0
                     : p.boundary == DRTS_OPEN ? 0.0
                     : fresnel(class_cos(c), p.media[k].n, p.n_outside);
            t.r_edge[k * 4 + c] = R;
            for (int k2 = 0; k2 < K; ++k2)
                t.r_int[(size_t(k) * K + k2) * 4 + c] = fresnel(class_cos(c), p.media[k].n, p.media[k2].n);
        }

    // exit fractions per (medium, face mask, direction)
    t.exit_total.assign(size_t(K) * 27 * kDirs, 0.0);
    t.exit_det.assign(size_t(K) * 27 * kDirs, 0.0);
    for (int k = 0; k < K; ++k) {
        const double *Wk = &t.W[size_t(k) * kDirs * kOffs * kDirs];
        for (int mask = 0; mask < 27; ++mask)
            for (int n = 0; n < kDirs; ++n) {
                const size_t ti = (size_t(k) * 27 + mask) * kDirs + n;
                column_exit(&Wk[size_t(n) * kOffs * kDirs], &t.r_edge[k * 4], mask, p.det_face,
                            t.exit_total[ti], t.exit_det[ti]);
            }
    }

    if (p.interface == DRTS_INTERFACE_TWO_STEP && path_frac == 1.0) {
        const std::string err = build_two_step_tables(p, t);
        if (!err.empty()) return err;
    } else {
        // one ledger class per medium
        t.n_classes = K;
        t.led_absorb = t.absorb;
        t.led_exit_total = t.exit_total;
        t.led_exit_det = t.exit_det;
    }
    return std::string();
}

}  // namespace drts
