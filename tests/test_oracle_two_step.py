"""Pins of the oracle's planar two-step interface crossing (Section 4.2,
reading R19: the path in medium 1 to the crossing point C, a Fresnel split at
the true incidence angle, the refracted direction by Snell's law shared
between the two lattice directions that bracket its polar angle, the rest of
the step in each medium as a Dirac source at C).  Every expected value below
is computed here from the geometry and textbook formulas, not from the
oracle:
  * mass: R + T = 1 with no absorption, the reflected share equal to the
    unpolarised Fresnel reflectance at the true angle;
  * Snell: the transmitted share splits between the two bracketing lattice
    directions so that the weighted polar angle equals the Snell angle;
  * a scattering-free beam lands around C + (1 - tc) L S (reflected and
    refracted) with the Eq. 18 weights (h - d) / sum;
  * normal incidence: R = ((n1 - n2) / (n1 + n2))^2, the beam keeps +z;
  * absorption along the two path pieces (closed form);
  * equal refractive indices: the option changes nothing;
  * mirror symmetry of a layered box, and layered media required.
No device."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1611_08536_gb300 import inputs as I


def layered(nz_low, nz_high, m_low, m_high, side=6, h=0.1, interface=1, boundary=I.MIRROR):
    nz = nz_low + nz_high
    mov = np.zeros((nz, side, side), np.uint8)
    mov[nz_low:] = 1
    return I.Problem((side, side, nz), h, [m_low, m_high], mov, n_outside=1.0, boundary=boundary,
                     precision=I.FP64, n_rhs=1, det_face=I.FACE_PZ, interface=interface)


def matrix(oracle_mod, prob):
    A = oracle_mod.assemble(prob)
    n = prob.n_states
    return sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(n, n))


DIRV = [I.direction_vector(d) for d in range(26)]


def dir_index(v):
    return DIRV.index(tuple(v))


def column(M, prob, voxel, d):
    nx, ny, _ = prob.shape
    x, y, z = voxel
    s = ((z * ny + y) * nx + x) * 26 + d
    c = M.getcol(s).tocoo()
    out = {}
    for r, w in zip(c.row, c.data):
        v, m = divmod(int(r), 26)
        out[(v % nx, v // nx % ny, v // (nx * ny), m)] = float(w)
    return out


def fresnel(cos_i, n1, n2):
    sin_t = n1 / n2 * math.sqrt(1 - cos_i * cos_i)
    if sin_t >= 1:
        return 1.0
    cos_t = math.sqrt(1 - sin_t * sin_t)
    rs = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t)
    rp = (n1 * cos_t - n2 * cos_i) / (n1 * cos_t + n2 * cos_i)
    return 0.5 * (rs * rs + rp * rp)


def point_weights(B):
    """Eq. 18: lattice offsets closer than 1 (units of h) to B, weights (1 - d) / sum."""
    pts = {}
    for z in range(-2, 3):
        for y in range(-2, 3):
            for x in range(-2, 3):
                d = math.dist((x, y, z), B)
                if d * d < 1 - 1e-9:
                    pts[(x, y, z)] = 1 - d
    s = sum(pts.values())
    return {k: v / s for k, v in pts.items()}


SRC = (2, 2, 2)           # the last layer below the plane z = 2.5 (units of h)
OBLIQUE = dir_index((1, 0, 1))


def test_mass_and_fresnel_share_oblique(oracle_mod):
    n1, n2 = 1.0, 1.5
    prob = layered(3, 3, (0.0, 0.0, 0.0, n1), (0.0, 0.0, 0.0, n2))
    col = column(matrix(oracle_mod, prob), prob, SRC, OBLIQUE)
    assert sum(col.values()) == pytest.approx(1.0, abs=1e-13)           # R + T = 1
    nr = dir_index((1, 0, -1))
    refl = sum(w for k, w in col.items() if k[3] == nr)
    assert refl == pytest.approx(fresnel(1 / math.sqrt(2), n1, n2), rel=1e-12)


def test_snell_angle_of_the_transmitted_split(oracle_mod):
    n1, n2 = 1.0, 1.5
    prob = layered(3, 3, (0.0, 0.0, 0.0, n1), (0.0, 0.0, 0.0, n2))
    col = column(matrix(oracle_mod, prob), prob, SRC, OBLIQUE)
    t_n = sum(w for k, w in col.items() if k[3] == OBLIQUE)               # 45 degrees
    t_z = sum(w for k, w in col.items() if k[3] == dir_index((0, 0, 1)))  # 0 degrees
    T = 1 - fresnel(1 / math.sqrt(2), n1, n2)
    assert t_n + t_z == pytest.approx(T, rel=1e-12)
    theta_t = math.asin(n1 / n2 * math.sin(math.pi / 4))
    mean_angle = (t_n * math.pi / 4 + t_z * 0.0) / T
    assert mean_angle == pytest.approx(theta_t, rel=1e-12)
    # nothing else: no horizontal share when the refracted ray bends towards the normal
    assert all(k[3] in (OBLIQUE, dir_index((0, 0, 1)), dir_index((1, 0, -1))) for k in col)


def test_scattering_free_beam_lands_around_the_two_step_points(oracle_mod):
    n1, n2 = 1.0, 1.5
    prob = layered(3, 3, (0.0, 0.0, 0.0, n1), (0.0, 0.0, 0.0, n2))
    col = column(matrix(oracle_mod, prob), prob, SRC, OBLIQUE)
    lam1, lam2 = 1.0, n1 / n2                        # path per step / h (n_min = n1)
    s = 1 / math.sqrt(2)
    tc = 0.5 / (lam1 * s)
    C = (tc * lam1 * s, 0.0, tc * lam1 * s)          # on the plane z = 0.5 above the source
    assert C[2] == pytest.approx(0.5)
    R = fresnel(s, n1, n2)
    # reflected: along (1, 0, -1)/sqrt(2) for (1 - tc) lam1
    Br = (C[0] + (1 - tc) * lam1 * s, 0.0, C[2] - (1 - tc) * lam1 * s)
    nr = dir_index((1, 0, -1))
    exp_r = {(SRC[0] + o[0], SRC[1] + o[1], SRC[2] + o[2], nr): R * w for o, w in point_weights(Br).items()}
    got_r = {k: w for k, w in col.items() if k[3] == nr}
    assert set(got_r) == set(exp_r)
    for k in exp_r:
        assert got_r[k] == pytest.approx(exp_r[k], rel=1e-12)
    # refracted: Snell direction for (1 - tc) lam2, shared between +z and (1,0,1)
    th_t = math.asin(n1 / n2 * s)
    Bt = (C[0] + (1 - tc) * lam2 * math.sin(th_t), 0.0, C[2] + (1 - tc) * lam2 * math.cos(th_t))
    T = 1 - R
    w_n = th_t / (math.pi / 4)
    for d, share in ((OBLIQUE, w_n), (dir_index((0, 0, 1)), 1 - w_n)):
        exp_t = {(SRC[0] + o[0], SRC[1] + o[1], SRC[2] + o[2], d): T * share * w for o, w in point_weights(Bt).items()}
        got_t = {k: w for k, w in col.items() if k[3] == d}
        assert set(got_t) == set(exp_t), d
        for k in exp_t:
            assert got_t[k] == pytest.approx(exp_t[k], rel=1e-12)


def test_normal_incidence(oracle_mod):
    n1, n2 = 1.33, 1.5
    prob = layered(3, 3, (0.0, 0.0, 0.0, n1), (0.0, 0.0, 0.0, n2))
    up = dir_index((0, 0, 1))
    col = column(matrix(oracle_mod, prob), prob, SRC, up)
    R = ((n1 - n2) / (n1 + n2)) ** 2
    down = dir_index((0, 0, -1))
    assert sum(w for k, w in col.items() if k[3] == down) == pytest.approx(R, rel=1e-12)
    assert sum(w for k, w in col.items() if k[3] == up) == pytest.approx(1 - R, rel=1e-12)
    assert all(k[3] in (up, down) for k in col)
    lam1, lam2 = 1.0, n1 / n2
    tc = 0.5 / lam1
    Bt = (0.0, 0.0, tc * lam1 + (1 - tc) * lam2)
    exp_t = {(SRC[0] + o[0], SRC[1] + o[1], SRC[2] + o[2], up): (1 - R) * w for o, w in point_weights(Bt).items()}
    got_t = {k: w for k, w in col.items() if k[3] == up}
    assert set(got_t) == set(exp_t)
    for k in exp_t:
        assert got_t[k] == pytest.approx(exp_t[k], rel=1e-12)


def test_absorption_along_the_two_path_pieces(oracle_mod):
    n1, n2, h = 1.0, 1.5, 0.1
    mu_a1, mu_a2 = 0.3, 0.7
    prob = layered(3, 3, (0.0, mu_a1, 0.0, n1), (0.0, mu_a2, 0.0, n2), h=h)
    col = column(matrix(oracle_mod, prob), prob, SRC, OBLIQUE)
    lam1, lam2 = 1.0, n1 / n2
    s = 1 / math.sqrt(2)
    tc = 0.5 / (lam1 * s)
    R = fresnel(s, n1, n2)
    nr = dir_index((1, 0, -1))
    refl = sum(w for k, w in col.items() if k[3] == nr)
    trans = sum(w for k, w in col.items() if k[3] != nr)
    assert refl == pytest.approx(R * math.exp(-mu_a1 * lam1 * h), rel=1e-12)
    assert trans == pytest.approx((1 - R) * math.exp(-mu_a1 * tc * lam1 * h)
                                  * math.exp(-mu_a2 * (1 - tc) * lam2 * h), rel=1e-12)
    info = oracle_mod.column_info(prob)
    absorb = info[0] if isinstance(info, tuple) else info.absorb
    nx, ny, _ = prob.shape
    st = ((SRC[2] * ny + SRC[1]) * nx + SRC[0]) * 26 + OBLIQUE
    assert absorb[st] == pytest.approx(1 - refl - trans, rel=1e-12)


def test_scattering_conserves_mass_of_a_crossing_state(oracle_mod):
    prob = layered(3, 3, (12.0, 0.0, 0.9, 1.4), (6.0, 0.0, 0.7, 1.37))
    M = matrix(oracle_mod, prob)
    for d in (OBLIQUE, dir_index((0, 0, 1)), dir_index((1, 1, 1)), dir_index((-1, 1, 1))):
        assert sum(column(M, prob, SRC, d).values()) == pytest.approx(1.0, abs=1e-12), d


def test_equal_indices_make_the_option_inert(oracle_mod):
    a = layered(3, 3, (12.0, 0.01, 0.9, 1.4), (6.0, 0.03, 0.7, 1.4), interface=0)
    b = layered(3, 3, (12.0, 0.01, 0.9, 1.4), (6.0, 0.03, 0.7, 1.4), interface=1)
    Ma, Mb = matrix(oracle_mod, a), matrix(oracle_mod, b)
    assert np.array_equal(Ma.indptr, Mb.indptr) and np.array_equal(Ma.indices, Mb.indices)
    assert np.array_equal(Ma.data, Mb.data)


def test_layered_box_mirror_symmetry(oracle_mod):
    """Reflecting x -> nx - 1 - x maps the layered problem onto itself, so A
    commutes with the state permutation (voxel mirrored, dx reversed)."""
    prob = layered(3, 3, (12.0, 0.01, 0.9, 1.4), (6.0, 0.03, 0.7, 1.3))
    M = matrix(oracle_mod, prob)
    nx, ny, nz = prob.shape
    perm = np.empty(prob.n_states, np.int64)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for d in range(26):
                    dx, dy, dz = DIRV[d]
                    s = ((z * ny + y) * nx + x) * 26 + d
                    perm[s] = ((z * ny + y) * nx + (nx - 1 - x)) * 26 + dir_index((-dx, dy, dz))
    P = sp.csr_matrix((np.ones(prob.n_states), (perm, np.arange(prob.n_states))), shape=M.shape)
    D = (P @ M @ P.T - M).tocoo()
    assert np.abs(D.data).max(initial=0.0) < 1e-14


def test_two_step_needs_layered_media(oracle_mod):
    prob = layered(3, 3, (12.0, 0.01, 0.9, 1.4), (6.0, 0.03, 0.7, 1.3))
    prob.medium_of_voxel = prob.medium_of_voxel.copy()
    prob.medium_of_voxel[1, 2, 2] = 1                 # a voxel of the upper medium in a lower layer
    with pytest.raises(Exception):
        oracle_mod.assemble(prob)
