/*
 * DRTS oracle: a plain, slow FP64 CPU implementation of the Dynamic
 * Radiative Transfer System time step of Georgakopoulos, Politopoulos and
 * Georgiou (arXiv:1611.08536).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library) shares no code, header, table or constant with it.
 *
 * What it computes, in the paper's order:
 *   - absorption / scattering split of one time step, Eq. 2-10;
 *   - unscattered streaming to B = X + c dt S, Eq. 11, snapped to the
 *     lattice with the nearest-neighbour weights of Eq. 18;
 *   - single scattering S -> S' spread along the segment AB, Eq. 12 and
 *     the segment-distance weights of Eq. 19;
 *   - the element rule of Eq. 20-21 (w1, or w0 + w1 on the same direction);
 *   - the state vector of Eq. 22 and the system matrix of Eq. 23, built by
 *     scattering every source state's contributions into target rows;
 *   - boundary and interface reflection / refraction, Section 4.2, in the
 *     first-order reading stated at orc_fold(), or, for layered media, the
 *     two-step crossing of the planar interfaces (build_two_step());
 *   - the step J(t+dt) = A J(t) + B P(t) of Eq. 26 and the detector
 *     functional of Eq. 27 (exit mass through a face patch).
 *
 * Geometry (cubic lattice, 26 lattice directions):
 *   voxel v = (z*ny + y)*nx + x, position h*(x,y,z); sphere diameter 2dr = h.
 *   direction d enumerates {-1,0,1}^3 \ {0} with dz slowest and dx fastest.
 *   state s = v*26 + d (Eq. 22).
 *   dt = h / c_max, so the step length in medium k is L_k = h * n_min / n_k.
 *
 * Everything is FP64, round-to-nearest, compiled without FMA contraction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NDIR 26
/* Planted mistakes (test builds only, -DPLANT_...): the pin tests compile
 * the oracle with one of these and must fail.  None is set in normal builds. */
/* A lattice point is a nearest neighbour when its (squared, in units of h)
 * distance is below 1 by this margin: points exactly 2dr away are excluded
 * whatever the rounding of the evaluation (strict inequality of Eq. 18/19). */
#define TIE_MARGIN 1e-9

typedef struct {
    int32_t nx, ny, nz;
    double h;                 /* voxel size = 2 dr (mm) */
    int32_t n_media;
    const double *mu_s;       /* [n_media] 1/mm */
    const double *mu_a;       /* [n_media] 1/mm */
    const double *g;          /* [n_media] Henyey-Greenstein anisotropy */
    const double *n;          /* [n_media] refractive index */
    const uint8_t *medium;    /* [nx*ny*nz] medium of each voxel */
    double n_outside;         /* refractive index outside the grid */
    int32_t boundary;         /* 0 open, 1 mirror, 2 fresnel */
    int32_t det_face;         /* 0..5 = -x,+x,-y,+y,-z,+z; -1 for none */
    int32_t det_nu, det_nv;   /* detector patch grid on that face */
    int32_t interface;        /* 0 first-order folding (R6); 1 planar two-step (R19) */
    int32_t direction_weights; /* 0 every direction alike (R7); 1 quadrature shares (R7 variant) */
} orc_problem;

/* one raw contribution of a source state: target offset o, direction m */
typedef struct { int o[3]; int m; double w; } orc_entry;

typedef struct {
    int count[NDIR];
    orc_entry *e[NDIR];
} orc_stencil;

static int DIRV[NDIR][3];
static double DIRS[NDIR][3];
static int DIRI[27];          /* (dz+1)*9+(dy+1)*3+(dx+1) -> direction, -1 at 0 */

static void init_dirs(void)
{
    int d = 0;
    DIRI[13] = -1;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy && !dz) continue;
                DIRV[d][0] = dx; DIRV[d][1] = dy; DIRV[d][2] = dz;
                double len = sqrt((double)(dx * dx + dy * dy + dz * dz));
                DIRS[d][0] = dx / len; DIRS[d][1] = dy / len; DIRS[d][2] = dz / len;
                DIRI[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = d;
                ++d;
            }
}

int orc_direction(int d, int *out3)
{
    init_dirs();
    if (d < 0 || d >= NDIR) return -1;
    out3[0] = DIRV[d][0]; out3[1] = DIRV[d][1]; out3[2] = DIRV[d][2];
    return 0;
}

static double min_index(const orc_problem *P)
{
    double nmin = P->n[0];
    for (int k = 1; k < P->n_media; ++k) if (P->n[k] < nmin) nmin = P->n[k];
    return nmin;
}

/* distance (units of h) from lattice point p to the segment [a, b] */
static double seg_dist(const double p[3], const double a[3], const double b[3])
{
    double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    double ab2 = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
    double t = 0.0;
    if (ab2 > 0.0) {
        t = (ap[0] * ab[0] + ap[1] * ab[1] + ap[2] * ab[2]) / ab2;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
    }
    double q[3] = {a[0] + t * ab[0] - p[0], a[1] + t * ab[1] - p[1], a[2] + t * ab[2] - p[2]};
    return sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
}

/* Henyey-Greenstein phase value for cos(angle) = mu */
static double hg(double g, double mu)
{
#ifndef PLANT_HG_SIGN
    double den = 1.0 + g * g - 2.0 * g * mu;
#else
    double den = 1.0 + g * g + 2.0 * g * mu;
#endif
#ifndef PLANT_HG_EXPONENT
    return (1.0 - g * g) / (den * sqrt(den));
#else
    return (1.0 - g * g) / den;
#endif
}

/* Unpolarised Fresnel reflectance, Section 4.2 (reflection and refraction at a
 * change of refractive index), from the incidence cosine.  Total internal
 * reflection gives 1. */
double orc_fresnel(double cos_i, double n1, double n2)
{
    if (n1 == n2) return 0.0;
#ifdef PLANT_FRESNEL_SWAP
    { double tmp = n1; n1 = n2; n2 = tmp; }
#endif
    double sin_i = sqrt(1.0 - cos_i * cos_i);
    double sin_t = n1 / n2 * sin_i;
    if (sin_t >= 1.0) return 1.0;
    double cos_t = sqrt(1.0 - sin_t * sin_t);
    double rs = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t);
    double rp = (n1 * cos_t - n2 * cos_i) / (n1 * cos_t + n2 * cos_i);
    return 0.5 * (rs * rs + rp * rp);
}

/* Share of the unit sphere carried by lattice direction m when the kernel
 * weights directions as quadrature points (reading R7, variant): the unique
 * weights, equal within each class of the cube's symmetry (6 axes, 12 face
 * diagonals, 8 body diagonals), that integrate every polynomial of degree
 * <= 7 on the sphere exactly (odd ones vanish by the central symmetry).  Written from the class sizes and the sphere averages
 * <1> = 1, <x^2 y^2 z^2> = 1/105, <x^2 y^2> = 1/15 (solved in that order):
 * body diagonals (|x y z| = 1/sqrt(27)) carry 8 c / 27 = 1/105, face
 * diagonals (x^2 y^2 = 1/4 for 4 of 12) b + 8 c / 9 = 1/15, axes the rest. */
static double quadrature_share(int m)
{
    int k = (DIRV[m][0] != 0) + (DIRV[m][1] != 0) + (DIRV[m][2] != 0);
    double c = 27.0 / (8.0 * 105.0);
    double b = 1.0 / 15.0 - 8.0 * c / 9.0;
    double a = (1.0 - 12.0 * b - 8.0 * c) / 6.0;
    return k == 1 ? a : (k == 2 ? b : c);
}

static double direction_weight(int mode, int m)
{
    return mode == 1 ? quadrature_share(m) : 1.0;
}

/* Discrete Henyey-Greenstein kernel g(S_n, S_m), normalised over the 26
 * directions for each incoming n (the probability kernel of Eq. 1/19);
 * mode 1 weights each outgoing direction by its quadrature share. */
static void hg_table(double g, int mode, double G[NDIR][NDIR])
{
    for (int n = 0; n < NDIR; ++n) {
        double sum = 0.0;
        for (int m = 0; m < NDIR; ++m) {
            double mu = DIRS[n][0] * DIRS[m][0] + DIRS[n][1] * DIRS[m][1] + DIRS[n][2] * DIRS[m][2];
            G[n][m] = hg(g, mu);
            if (mode == 1) G[n][m] *= direction_weight(mode, m);
            sum += G[n][m];
        }
#ifndef PLANT_HG_UNNORMALISED
        for (int m = 0; m < NDIR; ++m) G[n][m] /= sum;
#else
        (void)sum;
#endif
    }
}

static void add_entry(orc_stencil *S, int n, int cap, const int o[3], int m, double w)
{
    orc_entry *E = S->e[n];
    for (int q = 0; q < S->count[n]; ++q)
        if (E[q].m == m && E[q].o[0] == o[0] && E[q].o[1] == o[1] && E[q].o[2] == o[2]) {
            E[q].w += w;            /* Eq. 21: w0 + w1 on the same direction */
            return;
        }
    if (S->count[n] >= cap) abort();
    E[S->count[n]].o[0] = o[0]; E[S->count[n]].o[1] = o[1]; E[S->count[n]].o[2] = o[2];
    E[S->count[n]].m = m; E[S->count[n]].w = w;
    S->count[n]++;
}

/* The raw (unfolded) contributions of every source direction n of one medium:
 * Eq. 18 (unscattered, target direction n) and Eq. 19 (scattered into every m),
 * combined by Eq. 21.  Offsets are searched over {-2..2}^3; a target outside
 * {-1,0,1}^3 cannot occur when L <= h and aborts (self-check). */
static int build_stencil_frac(const orc_problem *P, int k, double frac, orc_stencil *S)
{
    const int cap = 27 * NDIR;
    double lam = frac * min_index(P) / P->n[k];   /* path length / h */
    double L = lam * P->h;
    double surv_a = exp(-P->mu_a[k] * L);         /* Eq. 8 */
    double surv_s = exp(-P->mu_s[k] * L);         /* Eq. 3 */
    double f0 = surv_s * surv_a;                  /* Eq. 9 */
#ifdef PLANT_ABSORB_ONCE
    f0 = surv_s;                                  /* absorption dropped from N0 */
#endif
    double f1 = (1.0 - surv_s) * surv_a;          /* Eq. 10 */
    double G[NDIR][NDIR];
    hg_table(P->g[k], P->direction_weights, G);

    for (int n = 0; n < NDIR; ++n) {
        S->count[n] = 0;
        S->e[n] = (orc_entry *)malloc(sizeof(orc_entry) * cap);
        if (!S->e[n]) return -1;
        double B[3] = {lam * DIRS[n][0], lam * DIRS[n][1], lam * DIRS[n][2]};

        /* Eq. 18: unscattered population to the neighbours of B */
#ifdef PLANT_DROP_UNSCATTERED
        f0 = 0.0;
#endif
        if (f0 > 0.0) {
            double wsum = 0.0, wr[125]; int oo[125][3], cnt = 0;
            for (int z = -2; z <= 2; ++z) for (int y = -2; y <= 2; ++y) for (int x = -2; x <= 2; ++x) {
                double p[3] = {x, y, z};
                double dd = seg_dist(p, B, B);
                if (dd * dd < 1.0 - TIE_MARGIN) {
                    oo[cnt][0] = x; oo[cnt][1] = y; oo[cnt][2] = z;
                    wr[cnt] = 1.0 - dd; wsum += wr[cnt]; ++cnt;
                }
            }
            for (int q = 0; q < cnt; ++q) {
                if (abs(oo[q][0]) > 1 || abs(oo[q][1]) > 1 || abs(oo[q][2]) > 1) abort();
                add_entry(S, n, cap, oo[q], n, wr[q] / wsum * f0);
            }
        }
        /* Eq. 19: scattered population S_n -> S_m around the segment AB */
        if (f1 > 0.0) {
            for (int m = 0; m < NDIR; ++m) {
#ifdef PLANT_SEGMENT_SIGN
                double A[3] = {-lam * DIRS[m][0], -lam * DIRS[m][1], -lam * DIRS[m][2]};
#else
                double A[3] = {lam * DIRS[m][0], lam * DIRS[m][1], lam * DIRS[m][2]};
#endif
                double wsum = 0.0, wr[125]; int oo[125][3], cnt = 0;
                for (int z = -2; z <= 2; ++z) for (int y = -2; y <= 2; ++y) for (int x = -2; x <= 2; ++x) {
                    double p[3] = {x, y, z};
                    double dd = seg_dist(p, A, B);
                    if (dd * dd < 1.0 - TIE_MARGIN) {
                        oo[cnt][0] = x; oo[cnt][1] = y; oo[cnt][2] = z;
                        wr[cnt] = 1.0 - dd; wsum += wr[cnt]; ++cnt;
                    }
                }
                for (int q = 0; q < cnt; ++q) {
                    if (abs(oo[q][0]) > 1 || abs(oo[q][1]) > 1 || abs(oo[q][2]) > 1) abort();
                    add_entry(S, n, cap, oo[q], m, wr[q] / wsum * G[n][m] * f1);
                }
            }
        }
    }
    return 0;
}

/* the stencil of a whole step: path L_k = c_k dt */
static int build_stencil(const orc_problem *P, int k, orc_stencil *S)
{
    return build_stencil_frac(P, k, 1.0, S);
}

static void free_stencil(orc_stencil *S)
{
    for (int n = 0; n < NDIR; ++n) free(S->e[n]);
}

/* ------------------------------------------------------------------------ */
/* Planar interfaces crossed in two steps (Section 4.2; reading R19)         */

static inline int64_t vox(const orc_problem *P, int x, int y, int z);

/* Spread mass w over the lattice points closer than h to the segment [A, B]
 * (a point when A = B), weights (h - d) / sum (Eq. 18/19), into entries of
 * source direction n with target direction m. */
static void spread(orc_stencil *S, int n, int cap, const double A[3], const double B[3], int m, double w)
{
    if (!(w > 0.0)) return;
    double wsum = 0.0, wr[125];
    int oo[125][3], cnt = 0;
    for (int z = -2; z <= 2; ++z) for (int y = -2; y <= 2; ++y) for (int x = -2; x <= 2; ++x) {
        double p[3] = {x, y, z};
        double dd = seg_dist(p, A, B);
        if (dd * dd < 1.0 - TIE_MARGIN) {
            oo[cnt][0] = x; oo[cnt][1] = y; oo[cnt][2] = z;
            wr[cnt] = 1.0 - dd; wsum += wr[cnt]; ++cnt;
        }
    }
    for (int q = 0; q < cnt; ++q) {
        if (abs(oo[q][0]) > 1 || abs(oo[q][1]) > 1 || abs(oo[q][2]) > 1) abort();
        add_entry(S, n, cap, oo[q], m, wr[q] / wsum * w);
    }
}

/* A Dirac source of mass `mass` at point C (units of h) moving along unit
 * vector D for the path l (units of h) in a medium (mu_s, mu_a, phase row
 * grow[m] for scattering out of D): Eq. 18 for the unscattered share, landing
 * around C + l D in the directions dir[0..nd) with weights dw, Eq. 19 for the
 * scattered share around [C + l S_m, C + l D] into every m. */
static void dirac_step(orc_stencil *S, int n, int cap, const double C[3], const double D[3], double l,
                       double mu_s, double mu_a, double h, const double grow[NDIR], const int *dir,
                       const double *dw, int nd, double mass)
{
    double B[3] = {C[0] + l * D[0], C[1] + l * D[1], C[2] + l * D[2]};
    double un = mass * exp(-(mu_s + mu_a) * l * h);
    for (int q = 0; q < nd; ++q) spread(S, n, cap, B, B, dir[q], un * dw[q]);
    double sc = mass * (1.0 - exp(-mu_s * l * h)) * exp(-mu_a * l * h);
    if (sc > 0.0)
        for (int m = 0; m < NDIR; ++m) {
            double A[3] = {C[0] + l * DIRS[m][0], C[1] + l * DIRS[m][1], C[2] + l * DIRS[m][2]};
            spread(S, n, cap, A, B, m, sc * grow[m]);
        }
}

/*
 * Contributions of a source in medium k1 whose direction n reaches the plane
 * to a layer of medium k2 (another refractive index) half a voxel away, for
 * every n with S_nz != 0 and crossing fraction tc = 1/2 / (lambda_1 |S_nz|)
 * below 1 (active[n] = 1), split into entries that fold as usual (S1) and
 * entries that meet no further interface (S0):
 *  - S1: photons scattered before the crossing point, at a fraction s in
 *    [0, tc) of the step, land around the segment from lambda_1 S_m (s = 0)
 *    to lambda_1 (tc S_n + (1 - tc) S_m) (s = tc) in direction m, with the
 *    scattering probability of the path tc L_1 and the absorption of the
 *    whole step in medium 1 (Eq. 10 over the first part);
 *  - S0: the unscattered share exp(-(mu_s + mu_a) tc L_1) reaches C = tc L_1
 *    S_n and becomes two Dirac sources: R (unpolarised Fresnel at the true
 *    incidence angle) reflected along S_n with its z component reversed for
 *    the rest of the step in medium 1, 1 - R refracted by Snell's law for the
 *    rest of the step in medium 2 (path (1 - tc) L_2); the refracted
 *    direction's state is shared between the two lattice directions of its
 *    azimuth whose polar angles bracket its own, linearly in the angle (the
 *    normal +-z, the incident direction's angle, the horizontal).
 */
static int build_two_step(const orc_problem *P, int k1, int k2, orc_stencil *S1, orc_stencil *S0, int active[NDIR])
{
    const int cap = 27 * NDIR;
    double nmin = min_index(P), h = P->h;
    double n1 = P->n[k1], n2 = P->n[k2];
    double l1 = nmin / n1, l2 = nmin / n2;
    double G1[NDIR][NDIR];
    hg_table(P->g[k1], P->direction_weights, G1);
    for (int n = 0; n < NDIR; ++n) {
        S1->count[n] = S0->count[n] = 0;
        S1->e[n] = (orc_entry *)malloc(sizeof(orc_entry) * cap);
        S0->e[n] = (orc_entry *)malloc(sizeof(orc_entry) * cap);
        if (!S1->e[n] || !S0->e[n]) return -1;
        active[n] = 0;
        double sz = DIRS[n][2];
        if (sz == 0.0) continue;
        double tc = 0.5 / (l1 * fabs(sz));
        if (!(tc < 1.0)) continue;
        active[n] = 1;
        int sg = sz > 0.0 ? 1 : -1;
        /* scattered before C */
        double p1 = (1.0 - exp(-P->mu_s[k1] * tc * l1 * h)) * exp(-P->mu_a[k1] * l1 * h);
        if (p1 > 0.0)
            for (int m = 0; m < NDIR; ++m) {
                double A[3] = {l1 * DIRS[m][0], l1 * DIRS[m][1], l1 * DIRS[m][2]};
                double B[3];
                for (int a = 0; a < 3; ++a) B[a] = l1 * (tc * DIRS[n][a] + (1.0 - tc) * DIRS[m][a]);
                spread(S1, n, cap, A, B, m, p1 * G1[n][m]);
            }
        /* unscattered to C, then reflected and refracted */
        double p0 = exp(-(P->mu_s[k1] + P->mu_a[k1]) * tc * l1 * h);
        double C[3] = {tc * l1 * DIRS[n][0], tc * l1 * DIRS[n][1], tc * l1 * DIRS[n][2]};
        double cos_i = fabs(sz);
        double R = orc_fresnel(cos_i, n1, n2);
#ifdef PLANT_TWO_STEP_NO_FLIP
        int nr = n;
#else
        int nr = DIRI[(-DIRV[n][2] + 1) * 9 + (DIRV[n][1] + 1) * 3 + (DIRV[n][0] + 1)];
#endif
        double wr1 = 1.0;
        dirac_step(S0, n, cap, C, DIRS[nr], (1.0 - tc) * l1, P->mu_s[k1], P->mu_a[k1], h, G1[nr], &nr, &wr1, 1,
                   p0 * R);
        if (R < 1.0) {
            double sin_i = sqrt(1.0 - cos_i * cos_i);
#ifdef PLANT_SNELL_INVERTED
            double sin_t = n2 / n1 * sin_i;
            if (sin_t > 1.0) sin_t = 1.0;
#else
            double sin_t = n1 / n2 * sin_i;
#endif
            double cos_t = sqrt(1.0 - sin_t * sin_t);
            double D[3] = {0.0, 0.0, sg * cos_t};
            int dir[2];
            double dw[2];
            int nd = 1;
            dir[0] = n;
            dw[0] = 1.0;
            if (sin_i > 0.0) {
                double hl = sqrt(DIRS[n][0] * DIRS[n][0] + DIRS[n][1] * DIRS[n][1]);
                D[0] = sin_t * DIRS[n][0] / hl;
                D[1] = sin_t * DIRS[n][1] / hl;
                double th_i = atan2(sin_i, cos_i), th_t = atan2(sin_t, cos_t);
                int axis = DIRI[(sg + 1) * 9 + 1 * 3 + 1];
                int horiz = DIRI[1 * 9 + (DIRV[n][1] + 1) * 3 + (DIRV[n][0] + 1)];
                double half_pi = 2.0 * atan(1.0);
                if (th_t <= th_i) {
                    dir[0] = n;    dw[0] = th_t / th_i;
                    dir[1] = axis; dw[1] = 1.0 - dw[0];
                } else {
                    dir[0] = n;     dw[0] = (half_pi - th_t) / (half_pi - th_i);
                    dir[1] = horiz; dw[1] = 1.0 - dw[0];
                }
                nd = 2;
            }
            /* phase row for scattering out of the refracted direction */
            double grow[NDIR], gsum = 0.0;
            for (int m = 0; m < NDIR; ++m) {
                grow[m] = hg(P->g[k2], D[0] * DIRS[m][0] + D[1] * DIRS[m][1] + D[2] * DIRS[m][2]);
                if (P->direction_weights == 1) grow[m] *= direction_weight(1, m);
                gsum += grow[m];
            }
            for (int m = 0; m < NDIR; ++m) grow[m] /= gsum;
#ifdef PLANT_TWO_STEP_PATH_MEDIUM1
            dirac_step(S0, n, cap, C, D, (1.0 - tc) * l1, P->mu_s[k2], P->mu_a[k2], h, grow, dir, dw, nd,
                       p0 * (1.0 - R));
#else
            dirac_step(S0, n, cap, C, D, (1.0 - tc) * l2, P->mu_s[k2], P->mu_a[k2], h, grow, dir, dw, nd,
                       p0 * (1.0 - R));
#endif
        }
    }
    return 0;
}

/* Two-step tables of every ordered pair of media with different indices
 * (built on first use; NULL entries elsewhere). */
typedef struct {
    int K;
    orc_stencil *S1, *S0;    /* [K*K] */
    int *active;             /* [K*K][NDIR] */
    int *built;              /* [K*K] */
} orc_two_step;

static orc_two_step *two_step_new(const orc_problem *P)
{
    if (!P->interface) return NULL;
    orc_two_step *T = (orc_two_step *)calloc(1, sizeof(orc_two_step));
    int K = P->n_media;
    T->K = K;
    T->S1 = (orc_stencil *)calloc((size_t)K * K, sizeof(orc_stencil));
    T->S0 = (orc_stencil *)calloc((size_t)K * K, sizeof(orc_stencil));
    T->active = (int *)calloc((size_t)K * K * NDIR, sizeof(int));
    T->built = (int *)calloc((size_t)K * K, sizeof(int));
    return T;
}

static void two_step_free(orc_two_step *T)
{
    if (!T) return;
    for (int q = 0; q < T->K * T->K; ++q)
        if (T->built[q]) { free_stencil(&T->S1[q]); free_stencil(&T->S0[q]); }
    free(T->S1); free(T->S0); free(T->active); free(T->built); free(T);
}

/* The two-step tables for source (voxel i of medium k, direction n), or 0
 * when that state crosses no planar interface within the step. */
static int two_step_for(const orc_problem *P, orc_two_step *T, const int i[3], int k, int n,
                        const orc_stencil **S1, const orc_stencil **S0)
{
    if (!T || DIRV[n][2] == 0) return 0;
    int zn = i[2] + DIRV[n][2];
    if (zn < 0 || zn >= P->nz) return 0;
    int k2 = P->medium[vox(P, i[0], i[1], zn)];
    if (P->n[k2] == P->n[k]) return 0;
    int q = k * T->K + k2;
    if (!T->built[q]) {
        if (build_two_step(P, k, k2, &T->S1[q], &T->S0[q], T->active + (size_t)q * NDIR)) abort();
        T->built[q] = 1;
    }
    if (!T->active[(size_t)q * NDIR + n]) return 0;
    *S1 = &T->S1[q];
    *S0 = &T->S0[q];
    return 1;
}

static inline int64_t vox(const orc_problem *P, int x, int y, int z)
{
    return ((int64_t)z * P->ny + y) * P->nx + x;
}

static inline double nidx(const orc_problem *P, int x, int y, int z)
{
    return P->n[P->medium[vox(P, x, y, z)]];
}

/* cosine between lattice direction m and coordinate axis a */
static double axis_cos(int m, int a)
{
    return fabs(DIRS[m][a]);
}

typedef struct {
    int t[3];
    int m;
    double w;
} orc_out;

/*
 * Fold one raw contribution (source voxel i of medium k, raw target offset o,
 * target direction m, value w) into the grid.  Section 4.2 only outlines the
 * treatment of boundaries; this is its first-order reading:
 *
 *  - Domain edge.  A target outside the grid along axis a (x, then y, then z)
 *    is mirrored back across that face (index -1 -> 0, N -> N-1) with the
 *    direction component a reversed and keeps the fraction R; the rest
 *    (1 - R) leaves the medium through that face.  R = 1 for a mirror
 *    boundary, 0 for an open one, and the unpolarised Fresnel reflectance
 *    between the source medium and the outside for a Fresnel boundary, at
 *    the angle between the direction and the face normal.
 *  - Interface.  For a target inside the grid whose refractive index differs
 *    from the source voxel's, and only when no edge folding happened: the
 *    face normal is the first axis with a nonzero offset along which the
 *    source's axis-neighbour has a different index (else the first nonzero
 *    axis).  When the direction moves across that face, the Fresnel fraction
 *    R is reflected (target mirrored back to the source side along the
 *    normal, direction component reversed) and 1 - R is transmitted (same
 *    voxel, direction snapped to the same lattice direction).  The step uses
 *    the source medium throughout.
 *
 * Writes up to two in-grid outputs; exit[f] receives the mass that leaves
 * through face f = 2*axis + (high side).  no_interface skips the interface
 * part (the second part of a two-step crossing, which meets no further
 * interface within the step).
 */
static int orc_fold(const orc_problem *P, const int i[3], int k, const orc_entry *e,
                    orc_out out[2], double exit[6], int no_interface)
{
    int N[3] = {P->nx, P->ny, P->nz};
    int t[3] = {i[0] + e->o[0], i[1] + e->o[1], i[2] + e->o[2]};
    int dv[3] = {DIRV[e->m][0], DIRV[e->m][1], DIRV[e->m][2]};
    double w = e->w;
    int ghost = 0, nout = 0;

    for (int a = 0; a < 3; ++a) {
        if (t[a] >= 0 && t[a] < N[a]) continue;
        ghost = 1;
        double R;
        if (P->boundary == 1) R = 1.0;
        else if (P->boundary == 0) R = 0.0;
        else R = orc_fresnel(axis_cos(e->m, a), P->n[k], P->n_outside);
        int face = 2 * a + (t[a] >= N[a] ? 1 : 0);
        exit[face] += w * (1.0 - R);
        w *= R;
#ifdef PLANT_MIRROR_INDEX
        t[a] = t[a] < 0 ? 1 : N[a] - 2;
#else
        t[a] = t[a] < 0 ? 0 : N[a] - 1;
#endif
#ifdef PLANT_HIGH_FACE_NO_FLIP
        if (t[a] == 0) dv[a] = -dv[a];
#else
        dv[a] = -dv[a];
#endif
    }
    if (w == 0.0) return 0;

    if (!ghost && !no_interface && (e->o[0] || e->o[1] || e->o[2])) {
        double ni = P->n[k];
        double nt = nidx(P, t[0], t[1], t[2]);
        if (nt != ni) {
            int a = -1;
            for (int b = 0; b < 3 && a < 0; ++b) {
                if (!e->o[b]) continue;
                int nb[3] = {i[0], i[1], i[2]};
                nb[b] += e->o[b];
                if (nidx(P, nb[0], nb[1], nb[2]) != ni) a = b;
            }
            for (int b = 0; b < 3 && a < 0; ++b) if (e->o[b]) a = b;
            if (dv[a] * e->o[a] > 0) {
                double R = orc_fresnel(axis_cos(e->m, a), ni, nt);
                int tr[3] = {t[0], t[1], t[2]};
                tr[a] = i[a];
                int dr[3] = {dv[0], dv[1], dv[2]};
                dr[a] = -dr[a];
                if (w * R > 0.0) {
                    out[nout].t[0] = tr[0]; out[nout].t[1] = tr[1]; out[nout].t[2] = tr[2];
                    out[nout].m = DIRI[(dr[2] + 1) * 9 + (dr[1] + 1) * 3 + (dr[0] + 1)];
                    out[nout].w = w * R;
                    ++nout;
                }
                w *= (1.0 - R);
            }
        }
    }
    if (w > 0.0) {
        out[nout].t[0] = t[0]; out[nout].t[1] = t[1]; out[nout].t[2] = t[2];
        out[nout].m = DIRI[(dv[2] + 1) * 9 + (dv[1] + 1) * 3 + (dv[0] + 1)];
        out[nout].w = w;
        ++nout;
    }
    return nout;
}

/* ------------------------------------------------------------------------ */
/* CSR matrix of the rows whose voxel lies in planes [z0, z1)                */

typedef struct {
    int64_t n_rows, nnz, row0;   /* first row = canonical state index */
    int64_t *row_ptr;
    int32_t *col;
    double *val;
} orc_csr;

typedef struct { int32_t row; int32_t col; double val; } trip;

static int cmp_trip_col(const void *a, const void *b)
{
    const trip *x = (const trip *)a, *y = (const trip *)b;
    return (x->col > y->col) - (x->col < y->col);
}

static int check_problem(const orc_problem *P)
{
    if (P->nx < 2 || P->ny < 2 || P->nz < 2) return -1;
    if (P->n_media < 1 || P->n_media > 256) return -1;
    if ((int64_t)P->nx * P->ny * P->nz * NDIR >= ((int64_t)1 << 31)) return -1;
    for (int k = 0; k < P->n_media; ++k) if (P->n[k] <= 0.0) return -1;
    if (P->interface != 0 && P->interface != 1) return -1;
    if (P->interface == 1)              /* planar interfaces: one medium per z layer */
        for (int z = 0; z < P->nz; ++z) {
            int k0 = P->medium[vox(P, 0, 0, z)];
            for (int y = 0; y < P->ny; ++y) for (int x = 0; x < P->nx; ++x)
                if (P->medium[vox(P, x, y, z)] != k0) return -1;
        }
    return 0;
}

/* Assemble A's rows for voxel planes z in [z0, z1) (Eq. 20-23) by scattering
 * every source state of planes z0-1 .. z1 and keeping targets in range.  Rows
 * come out in canonical order, columns ascending, duplicates summed. */
orc_csr *orc_assemble(const orc_problem *P, int z0, int z1)
{
    init_dirs();
    if (check_problem(P) || z0 < 0 || z1 > P->nz || z0 >= z1) return NULL;
    orc_stencil *S = (orc_stencil *)calloc(P->n_media, sizeof(orc_stencil));
    for (int k = 0; k < P->n_media; ++k) build_stencil(P, k, &S[k]);
    orc_two_step *TS = two_step_new(P);

    int64_t plane_rows = (int64_t)P->nx * P->ny * NDIR;
    orc_csr *C = (orc_csr *)calloc(1, sizeof(orc_csr));
    C->row0 = vox(P, 0, 0, z0) * NDIR;
    C->n_rows = plane_rows * (z1 - z0);
    C->row_ptr = (int64_t *)malloc(sizeof(int64_t) * (C->n_rows + 1));
    C->row_ptr[0] = 0;
    int64_t cap = 0;

    int64_t tcap = plane_rows * 240;
    trip *T = (trip *)malloc(sizeof(trip) * tcap);
    trip *T2 = (trip *)malloc(sizeof(trip) * tcap);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (plane_rows + 1));

    for (int zt = z0; zt < z1; ++zt) {
        int64_t nt = 0;
        for (int zs = zt - 1; zs <= zt + 1; ++zs) {
            if (zs < 0 || zs >= P->nz) continue;
            for (int ys = 0; ys < P->ny; ++ys) for (int xs = 0; xs < P->nx; ++xs) {
                int i[3] = {xs, ys, zs};
                int k = P->medium[vox(P, xs, ys, zs)];
                for (int n = 0; n < NDIR; ++n) {
                    int32_t col = (int32_t)(vox(P, xs, ys, zs) * NDIR + n);
                    const orc_stencil *S1 = &S[k], *S0 = NULL;
                    two_step_for(P, TS, i, k, n, &S1, &S0);
                    int n1 = S1->count[n], n0 = S0 ? S0->count[n] : 0;
                    for (int q = 0; q < n1 + n0; ++q) {
                        orc_out out[2]; double ex[6] = {0};
                        int no = q < n1 ? orc_fold(P, i, k, &S1->e[n][q], out, ex, 0)
                                        : orc_fold(P, i, k, &S0->e[n][q - n1], out, ex, 1);
                        for (int u = 0; u < no; ++u) {
                            if (out[u].t[2] != zt) continue;
                            if (nt >= tcap) {
                                tcap *= 2;
                                T = (trip *)realloc(T, sizeof(trip) * tcap);
                                T2 = (trip *)realloc(T2, sizeof(trip) * tcap);
                            }
                            T[nt].row = (int32_t)(((int64_t)out[u].t[1] * P->nx + out[u].t[0]) * NDIR + out[u].m);
                            T[nt].col = col;
#ifdef PLANT_WRONG_DIRECTION_INDEX
                            T[nt].row = (int32_t)(((int64_t)out[u].t[1] * P->nx + out[u].t[0]) * NDIR
                                                  + (NDIR - 1 - out[u].m));
#endif
                            T[nt].val = out[u].w;
                            ++nt;
                        }
                    }
                }
            }
        }
        /* bucket by row, then sort each row by column and merge duplicates */
        memset(cnt, 0, sizeof(int64_t) * (plane_rows + 1));
        for (int64_t q = 0; q < nt; ++q) cnt[T[q].row + 1]++;
        for (int64_t r = 0; r < plane_rows; ++r) cnt[r + 1] += cnt[r];
        for (int64_t q = 0; q < nt; ++q) T2[cnt[T[q].row]++] = T[q];
        for (int64_t r = plane_rows; r > 0; --r) cnt[r] = cnt[r - 1];
        cnt[0] = 0;
        int64_t base = C->row_ptr[(zt - z0) * plane_rows];
        if (base + nt > cap) {
            cap = (base + nt) * 2 + 1024;
            C->col = (int32_t *)realloc(C->col, sizeof(int32_t) * cap);
            C->val = (double *)realloc(C->val, sizeof(double) * cap);
        }
        int64_t pos = base;
        for (int64_t r = 0; r < plane_rows; ++r) {
            trip *row = T2 + cnt[r];
            int64_t len = cnt[r + 1] - cnt[r];
            qsort(row, (size_t)len, sizeof(trip), cmp_trip_col);
            for (int64_t q = 0; q < len; ++q) {
                if (pos > base && q > 0 && C->col[pos - 1] == row[q].col) {
                    C->val[pos - 1] += row[q].val;
                } else {
                    C->col[pos] = row[q].col;
                    C->val[pos] = row[q].val;
                    ++pos;
                }
            }
            C->row_ptr[(zt - z0) * plane_rows + r + 1] = pos;
        }
    }
    C->nnz = C->row_ptr[C->n_rows];
    free(T); free(T2); free(cnt);
    for (int k = 0; k < P->n_media; ++k) free_stencil(&S[k]);
    free(S);
    two_step_free(TS);
    return C;
}

void orc_csr_info(const orc_csr *C, int64_t *n_rows, int64_t *nnz, int64_t *row0)
{
    *n_rows = C->n_rows; *nnz = C->nnz; *row0 = C->row0;
}

void orc_csr_copy(const orc_csr *C, int64_t *row_ptr, int32_t *col, double *val)
{
    memcpy(row_ptr, C->row_ptr, sizeof(int64_t) * (C->n_rows + 1));
    memcpy(col, C->col, sizeof(int32_t) * C->nnz);
    memcpy(val, C->val, sizeof(double) * C->nnz);
}

void orc_csr_free(orc_csr *C)
{
    if (!C) return;
    free(C->row_ptr); free(C->col); free(C->val); free(C);
}

/* Per-state column functionals.  absorb[s] = 1 - exp(-mu_a L) (Eq. 8),
 * exit_total[s] = mass of state s that leaves the grid in one step,
 * exit_det[s] = the part of it that leaves through the detector face,
 * det_patch[s] = detector patch of s's voxel (or -1).  Eq. 27 with F = exit. */
int orc_column_info(const orc_problem *P, double *absorb, double *exit_total,
                    double *exit_det, int32_t *det_patch)
{
    init_dirs();
    if (check_problem(P)) return -1;
    orc_stencil *S = (orc_stencil *)calloc(P->n_media, sizeof(orc_stencil));
    for (int k = 0; k < P->n_media; ++k) build_stencil(P, k, &S[k]);
    orc_two_step *TS = two_step_new(P);
    double nmin = min_index(P);
    int N[3] = {P->nx, P->ny, P->nz};
    int fa = P->det_face >= 0 ? P->det_face / 2 : -1;
    int ua = fa == 0 ? 1 : 0, va = fa == 2 ? 1 : 2;
    for (int z = 0; z < P->nz; ++z) for (int y = 0; y < P->ny; ++y) for (int x = 0; x < P->nx; ++x) {
        int i[3] = {x, y, z};
        int64_t v = vox(P, x, y, z);
        int k = P->medium[v];
        double L = nmin / P->n[k] * P->h;
        int patch = -1;
        if (fa >= 0) {
            int on = (P->det_face & 1) ? (i[fa] == N[fa] - 1) : (i[fa] == 0);
            if (on) patch = (int)((int64_t)i[va] * P->det_nv / N[va]) * P->det_nu
                            + (int)((int64_t)i[ua] * P->det_nu / N[ua]);
        }
        for (int n = 0; n < NDIR; ++n) {
            double ex[6] = {0, 0, 0, 0, 0, 0};
            const orc_stencil *S1 = &S[k], *S0 = NULL;
            two_step_for(P, TS, i, k, n, &S1, &S0);
            for (int q = 0; q < S1->count[n]; ++q) {
                orc_out out[2];
                orc_fold(P, i, k, &S1->e[n][q], out, ex, 0);
            }
            for (int q = 0; S0 && q < S0->count[n]; ++q) {
                orc_out out[2];
                orc_fold(P, i, k, &S0->e[n][q], out, ex, 1);
            }
            int64_t s = v * NDIR + n;
            absorb[s] = 1.0 - exp(-P->mu_a[k] * L);
            if (S0) {   /* a two-step crossing: whatever the raw entries do not carry is absorbed */
                double kept = 0.0;
                for (int q = 0; q < S1->count[n]; ++q) kept += S1->e[n][q].w;
                for (int q = 0; q < S0->count[n]; ++q) kept += S0->e[n][q].w;
                absorb[s] = 1.0 - kept;
            }
            exit_total[s] = ex[0] + ex[1] + ex[2] + ex[3] + ex[4] + ex[5];
            exit_det[s] = P->det_face >= 0 ? ex[P->det_face] : 0.0;
            det_patch[s] = patch;
        }
    }
    for (int k = 0; k < P->n_media; ++k) free_stencil(&S[k]);
    free(S);
    two_step_free(TS);
    return 0;
}

/* y = A x for the rows of C (x indexed by canonical state, y by local row) */
void orc_spmv(const orc_csr *C, const double *x, double *y, int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t r = 0; r < C->n_rows; ++r) {
        double acc = 0.0;
        for (int64_t q = C->row_ptr[r]; q < C->row_ptr[r + 1]; ++q) acc += C->val[q] * x[C->col[q]];
        y[r] = acc;
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Run n_steps of Eq. 26 from x (in place) on a full-grid CSR:
 *   for t in [t_begin, t_begin + n_steps):
 *     det[t - t_begin][p] = sum of exit_det[s] x_t[s] over s in patch p  (Eq. 27)
 *     ledger: absorbed += absorb . x_t, exited += exit_total . x_t
 *     x_{t+1} = A x_t + s(t),  s(t) = sum_e w_e P(t) e_{state_e}
 * P(t) = profile[t - t0] for t0 <= t < t0 + n_t, else 0.
 * ledger[4] = {sum x at the end, injected, absorbed, exited} (accumulated).
 * Optional sparse detector rows (Eq. 27 with a general F: point detectors,
 * chosen (voxel, direction) states): fdet[t - t_begin][d] = sum over entries
 * e with fe_det[e] = d of fe_w[e] x_t[fe_state[e]], in entry order.
 */
int orc_run(const orc_csr *C, double *x, int64_t t_begin, int64_t n_steps,
            int32_t n_src, const int64_t *src_state, const double *src_w,
            int64_t t0, int32_t n_t, const double *profile,
            const double *absorb, const double *exit_total, const double *exit_det,
            const int32_t *det_patch, int32_t n_patch, double *det, double *ledger,
            int64_t n_fe, const int32_t *fe_det, const int64_t *fe_state, const double *fe_w,
            int32_t n_fdet, double *fdet, int n_threads)
{
    if (C->row0 != 0) return -1;
    int64_t n = C->n_rows;
    for (int64_t e = 0; e < n_fe; ++e)
        if (fe_det[e] < 0 || fe_det[e] >= n_fdet || fe_state[e] < 0 || fe_state[e] >= n) return -3;
    double *y = (double *)malloc(sizeof(double) * n);
    if (!y) return -2;
    for (int64_t t = t_begin; t < t_begin + n_steps; ++t) {
        double *dt = det ? det + (t - t_begin) * n_patch : NULL;
        if (dt) for (int p = 0; p < n_patch; ++p) dt[p] = 0.0;
        /* sparse detector rows F of Eq. 27: one weighted sum of x_t per detector */
        if (fdet) {
            double *ft = fdet + (t - t_begin) * n_fdet;
            for (int32_t d = 0; d < n_fdet; ++d) ft[d] = 0.0;
            for (int64_t e = 0; e < n_fe; ++e) {
#ifdef PLANT_POINT_OFF_BY_ONE
                ft[fe_det[e]] += fe_w[e] * x[fe_state[e] > 0 ? fe_state[e] - 1 : 0];
#else
                ft[fe_det[e]] += fe_w[e] * x[fe_state[e]];
#endif
            }
        }
        double ab = 0.0, ex = 0.0;
        for (int64_t s = 0; s < n; ++s) {
            ab += absorb[s] * x[s];
            ex += exit_total[s] * x[s];
            if (dt && det_patch[s] >= 0) dt[det_patch[s]] += exit_det[s] * x[s];
        }
        ledger[2] += ab;
        ledger[3] += ex;
        orc_spmv(C, x, y, n_threads);
        if (t >= t0 && t < t0 + n_t) {
            for (int32_t e = 0; e < n_src; ++e) {
                double inj = src_w[e] * profile[t - t0];
                y[src_state[e]] += inj;
                ledger[1] += inj;
            }
        }
        memcpy(x, y, sizeof(double) * n);
    }
    double sum = 0.0;
    for (int64_t s = 0; s < n; ++s) sum += x[s];
    ledger[0] = sum;
    free(y);
    return 0;
}

/* Dense raw stencil of one medium, W[n][o][m] with o = (oz+1)*9+(oy+1)*3+(ox+1),
 * before any folding (test access to Eq. 18/19/21 values). */
int orc_raw_stencil(const orc_problem *P, int k, double *W)
{
    init_dirs();
    if (check_problem(P) || k < 0 || k >= P->n_media) return -1;
    orc_stencil S;
    build_stencil(P, k, &S);
    memset(W, 0, sizeof(double) * NDIR * 27 * NDIR);
    for (int n = 0; n < NDIR; ++n)
        for (int q = 0; q < S.count[n]; ++q) {
            const orc_entry *e = &S.e[n][q];
            int o = (e->o[2] + 1) * 9 + (e->o[1] + 1) * 3 + (e->o[0] + 1);
            W[((int64_t)n * 27 + o) * NDIR + e->m] += e->w;
        }
    free_stencil(&S);
    return 0;
}

/* Dense two-step entries of a source in medium k1 next to a z layer of
 * medium k2 (another refractive index): S1[n][o][m] (folded like the usual
 * entries), S0[n][o][m] (folded at the grid edge only) and active[n] (S_n
 * reaches the plane within the step); test access to build_two_step(). */
int orc_two_step_stencil(const orc_problem *P, int k1, int k2, double *S1, double *S0, int32_t *active)
{
    init_dirs();
    if (check_problem(P) || k1 < 0 || k1 >= P->n_media || k2 < 0 || k2 >= P->n_media) return -1;
    if (P->n[k1] == P->n[k2]) return -1;
    orc_stencil A, B;
    int act[NDIR];
    if (build_two_step(P, k1, k2, &A, &B, act)) return -1;
    memset(S1, 0, sizeof(double) * NDIR * 27 * NDIR);
    memset(S0, 0, sizeof(double) * NDIR * 27 * NDIR);
    for (int n = 0; n < NDIR; ++n) {
        active[n] = act[n];
        for (int q = 0; q < A.count[n]; ++q) {
            const orc_entry *e = &A.e[n][q];
            int o = (e->o[2] + 1) * 9 + (e->o[1] + 1) * 3 + (e->o[0] + 1);
            S1[((int64_t)n * 27 + o) * NDIR + e->m] += e->w;
        }
        for (int q = 0; q < B.count[n]; ++q) {
            const orc_entry *e = &B.e[n][q];
            int o = (e->o[2] + 1) * 9 + (e->o[1] + 1) * 3 + (e->o[0] + 1);
            S0[((int64_t)n * 27 + o) * NDIR + e->m] += e->w;
        }
    }
    free_stencil(&A);
    free_stencil(&B);
    return 0;
}

/*
 * Sensor response of Eq. 27: a sensor integrates the photons reaching it with
 * an impulse response h over a window of +-w steps around t,
 *   M[t][d] = sum over k in [t - w, t + w], 0 <= k < T, of h[t - k + w] D[k][d],
 * where D[k][d] is the detector readout of step k (the F-weighted photon count
 * of x_k) and h[j + w] the response at lag j (in steps).
 */
void orc_sensor_response(const double *D, int64_t T, int32_t n_det, int32_t w, const double *h,
                         double *M)
{
    for (int64_t t = 0; t < T; ++t)
        for (int32_t d = 0; d < n_det; ++d) {
            double acc = 0.0;
            for (int64_t k = t - w; k <= t + w; ++k) {
                if (k < 0 || k >= T) continue;
#ifdef PLANT_SENSOR_LAG_SIGN
                acc += h[k - t + w] * D[k * n_det + d];
#else
                acc += h[t - k + w] * D[k * n_det + d];
#endif
            }
            M[t * n_det + d] = acc;
        }
}

/*
 * Column of the source matrix B of Eq. 26 for photons emitted during a step
 * (Section 4.1: the source function is partitioned in time within the step).
 * A unit population leaves the centre of voxel i in direction n and travels
 * the fraction frac of the step's path L_k before the step ends: the same
 * absorption / scattering split and lattice weights as the system matrix
 * (Eq. 18, 19, 21) with the path frac * L_k, folded at the domain edge and at
 * interfaces the same way.  frac = 1 gives column (i, n) of A; frac -> 0
 * leaves the unit population in state (i, n).
 * Writes the distinct target states in ascending order with their values;
 * returns their count (or -1 on bad input, -2 if cap is too small) and the
 * mass that leaves the grid in exit_mass.
 */
int orc_source_column(const orc_problem *P, int64_t state, double frac, int32_t cap,
                      int64_t *out_state, double *out_w, double *exit_mass)
{
    init_dirs();
    if (check_problem(P) || frac <= 0.0 || frac > 1.0) return -1;
    int64_t V = (int64_t)P->nx * P->ny * P->nz;
    if (state < 0 || state >= V * NDIR) return -1;
    int64_t v = state / NDIR;
    int n = (int)(state % NDIR);
    int i[3] = {(int)(v % P->nx), (int)(v / P->nx % P->ny), (int)(v / ((int64_t)P->nx * P->ny))};
    int k = P->medium[v];
    orc_stencil S;
#ifdef PLANT_SOURCE_FULL_PATH
    frac = 1.0;
#endif
    if (build_stencil_frac(P, k, frac, &S)) return -1;
    int64_t tcap = 2 * (int64_t)S.count[n] + 1;
    int64_t *ts = (int64_t *)malloc(sizeof(int64_t) * tcap);
    double *tw = (double *)malloc(sizeof(double) * tcap);
    int64_t nt = 0;
    double ex[6] = {0, 0, 0, 0, 0, 0};
    for (int q = 0; q < S.count[n]; ++q) {
        orc_out out[2];
        int no = orc_fold(P, i, k, &S.e[n][q], out, ex, 0);
        for (int u = 0; u < no; ++u) {
            ts[nt] = vox(P, out[u].t[0], out[u].t[1], out[u].t[2]) * NDIR + out[u].m;
            tw[nt] = out[u].w;
            ++nt;
        }
    }
    /* insertion sort by target state (stable), then merge equal targets */
    for (int64_t a = 1; a < nt; ++a) {
        int64_t sk = ts[a]; double wk = tw[a]; int64_t b = a - 1;
        while (b >= 0 && ts[b] > sk) { ts[b + 1] = ts[b]; tw[b + 1] = tw[b]; --b; }
        ts[b + 1] = sk; tw[b + 1] = wk;
    }
    int64_t cnt = 0;
    for (int64_t a = 0; a < nt; ++a) {
        if (cnt > 0 && ts[a] == out_state[cnt - 1]) { out_w[cnt - 1] += tw[a]; continue; }
        if (cnt >= cap) { cnt = -2; break; }
        out_state[cnt] = ts[a];
        out_w[cnt] = tw[a];
        ++cnt;
    }
    if (exit_mass) *exit_mass = ex[0] + ex[1] + ex[2] + ex[3] + ex[4] + ex[5];
    free(ts); free(tw);
    free_stencil(&S);
    return (int)cnt;
}
