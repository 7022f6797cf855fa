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

}  // namespace

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
            double phase[kDirs], psum = 0.0;
            for (int m = 0; m < kDirs; ++m) {
                double mu = D.u[n][0] * D.u[m][0] + D.u[n][1] * D.u[m][1] + D.u[n][2] * D.u[m][2];
                double den = 1.0 + md.g * md.g - 2.0 * md.g * mu;
                phase[m] = (1.0 - md.g * md.g) / (den * std::sqrt(den));
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

    // exit fractions per (medium, face mask, direction): a raw target outside
    // the grid along axis a (x, then y, then z) keeps R and lets 1 - R out
    // through that face (Section 4.2 edge reading)
    t.exit_total.assign(size_t(K) * 27 * kDirs, 0.0);
    t.exit_det.assign(size_t(K) * 27 * kDirs, 0.0);
    for (int k = 0; k < K; ++k) {
        const double *Wk = &t.W[size_t(k) * kDirs * kOffs * kDirs];
        for (int mask = 0; mask < 27; ++mask) {
            const int b[3] = {mask % 3, mask / 3 % 3, mask / 9};
            for (int n = 0; n < kDirs; ++n) {
                double tot = 0.0, det = 0.0;
                for (int o = 0; o < kOffs; ++o) {
                    const int ov[3] = {o % 3 - 1, o / 3 % 3 - 1, o / 9 - 1};
                    for (int m = 0; m < kDirs; ++m) {
                        double w = Wk[(n * kOffs + o) * kDirs + m];
                        if (w <= 0.0) continue;
                        for (int a = 0; a < 3; ++a) {
                            const bool out_lo = b[a] == 0 && ov[a] == -1;
                            const bool out_hi = b[a] == 2 && ov[a] == 1;
                            if (!out_lo && !out_hi) continue;
                            const int c = D.v[m][a] != 0 ? D.nnzc[m] : 0;
                            const double R = t.r_edge[k * 4 + c];
                            const double leave = w * (1.0 - R);
                            tot += leave;
                            if (p.det_face == 2 * a + (out_hi ? 1 : 0)) det += leave;
                            w *= R;
                        }
                    }
                }
                t.exit_total[(size_t(k) * 27 + mask) * kDirs + n] = tot;
                t.exit_det[(size_t(k) * 27 + mask) * kDirs + n] = det;
            }
        }
    }
    return std::string();
}

}  // namespace drts
