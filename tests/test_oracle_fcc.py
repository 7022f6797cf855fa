"""Pins of the close-packed (FCC) sphere-partition oracle (Section 3 of
arXiv:1611.08536, Eq. 18-26) against what the method fixes: closed-form
targets and weights, Eq. 24 column sums, the symmetry of the packing,
ballistic translation, pure absorption decay, ledger closure, and dense
matrix powers from a loop-literal transcription on a small box."""
import itertools
import math

import numpy as np
import pytest

from oracle import fcc

S2 = math.sqrt(2.0)


def _opposite(n, offs):
    return int(np.flatnonzero((offs == -offs[n]).all(axis=1))[0])


def test_lattice_and_directions():
    offs = fcc.neighbour_offsets()
    assert offs.shape == (12, 3)
    assert np.all((offs ** 2).sum(axis=1) == 2)               # touching spheres, distance s
    assert len({tuple(o) for o in offs}) == 12
    assert np.allclose(np.linalg.norm(fcc.directions(), axis=1), 1.0, rtol=0, atol=1e-15)
    C = fcc.site_coords((6, 4, 5))
    assert len(C) == 6 * 4 * 5 // 2 and np.all(C.sum(axis=1) % 2 == 0)
    assert [fcc.site_index((6, 4, 5), c) for c in C] == list(range(len(C)))


def test_unscattered_lattice_direction_lands_on_one_neighbour():
    # mu_s = 0, L = s: B is the neighbour's centre, every other site is at
    # least s away, so Eq. 18 gives one target of weight 1
    W = fcc.stencil(0.0, 0.0, 0.9, 1.0, 0.1)
    offs = fcc.neighbour_offsets()
    assert len(W) == 12
    for n in range(12):
        assert W[(n, tuple(int(v) for v in offs[n]), n)] == 1.0


def test_opposite_direction_segment_closed_form():
    # Scattering from S_n into -S_n: the segment A_m B runs from -off_n to
    # +off_n through the source centre.  Sites closer than s = sqrt(2) a:
    # the centre and both ends (distance 0, weight sqrt 2) and the eight
    # sites (+-1, 0, +-1)-type with projection +-1/sqrt 2 and perpendicular
    # distance sqrt(3/2) (weight sqrt 2 - sqrt 1.5); (1, -1, 0)-type sites sit
    # exactly at s and are excluded.
    mu_s, s_mm = 1000.0, 0.1                   # unscattered share e^-100: negligible
    W = fcc.stencil(mu_s, 0.0, 0.0, 1.0, s_mm)
    offs = fcc.neighbour_offsets()
    sc = (1.0 - math.exp(-mu_s * s_mm)) / 12.0  # g = 0: G = 1/12
    total = 3 * S2 + 8 * (S2 - math.sqrt(1.5))
    for n in range(12):
        m = _opposite(n, offs)
        got = {off: v for (nn, off, mm), v in W.items() if nn == n and mm == m}
        assert len(got) == 11
        heavy = {(0, 0, 0), tuple(int(v) for v in offs[n]), tuple(int(-v) for v in offs[n])}
        for off, v in got.items():
            want = (S2 if off in heavy else S2 - math.sqrt(1.5)) / total * sc
            assert v == pytest.approx(want, rel=1e-14, abs=0)
        light = [np.array(o) for o in got if o not in heavy]
        u = offs[n] / S2
        for o in light:
            assert abs(o @ u) == pytest.approx(1 / S2, rel=1e-15)
            assert (o @ o) - (o @ u) ** 2 == pytest.approx(1.5, rel=1e-15)


@pytest.mark.parametrize("mu_s,mu_a,g", [(10.0, 0.01, 0.9), (3.0, 0.5, 0.0), (25.0, 0.1, 0.7), (0.0, 0.2, 0.5)])
def test_column_sums_eq24(mu_s, mu_a, g):
    s_mm = 0.1
    W = fcc.stencil(mu_s, mu_a, g, 1.0, s_mm)
    tot = np.zeros(12)
    for (n, _o, _m), v in W.items():
        assert v > 0.0
        tot[n] += v
    assert np.allclose(tot, math.exp(-mu_a * s_mm), rtol=1e-14, atol=0)


def test_isotropic_scattering_is_uniform_over_directions():
    mu_s, mu_a, s_mm = 8.0, 0.3, 0.1
    W = fcc.stencil(mu_s, mu_a, 0.0, 1.0, s_mm)
    into = np.zeros((12, 12))
    for (n, _o, m), v in W.items():
        into[n, m] += v
    sc = (1.0 - math.exp(-mu_s * s_mm)) * math.exp(-mu_a * s_mm) / 12.0
    un = math.exp(-mu_s * s_mm) * math.exp(-mu_a * s_mm)
    assert np.allclose(into, sc + np.eye(12) * un, rtol=1e-14, atol=0)


def _signed_permutations():
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            P = np.zeros((3, 3), dtype=np.int64)
            for r in range(3):
                P[r, perm[r]] = signs[r]
            yield P


def test_stencil_respects_the_symmetry_of_the_packing():
    # every rotation or reflection of the cube maps the packing, the
    # direction set and so the transitions onto themselves
    W = fcc.stencil(12.0, 0.05, 0.85, 1.0, 0.1)
    offs = fcc.neighbour_offsets()
    index = {tuple(o): i for i, o in enumerate(offs)}
    groups = list(_signed_permutations())
    assert len(groups) == 48
    for P in groups:
        dmap = [index[tuple(P @ o)] for o in offs]
        for (n, off, m), v in W.items():
            key = (dmap[n], tuple(int(c) for c in P @ np.array(off)), dmap[m])
            assert W[key] == pytest.approx(v, rel=1e-13, abs=0)


def _problem(shape, media, medium=None, s_mm=0.1):
    n_sites = shape[0] * shape[1] * shape[2] // 2
    if medium is None:
        medium = np.zeros(n_sites, np.uint8)
    return fcc.FccProblem(shape, s_mm, media, medium)


def test_ballistic_translation_and_exit():
    prob = _problem((10, 10, 10), [(0.0, 0.0, 0.9, 1.4)])
    A, ex = fcc.assemble(prob)
    offs = fcc.neighbour_offsets()
    n = int(np.flatnonzero((offs == [1, 0, 1]).all(axis=1))[0])
    c0 = np.array([1, 4, 1])
    st = fcc.site_index(prob.shape, c0) * 12 + n
    for t in range(1, 12):
        x, led = fcc.run(A, t, [st], [1.0], [1.0], absorb=fcc.absorb_fraction(prob), exit_frac=ex)
        c = c0 + (t - 1) * offs[n]
        if np.all(c < 10):
            want = np.zeros_like(x)
            want[fcc.site_index(prob.shape, c) * 12 + n] = 1.0
            assert np.array_equal(x, want)
        else:
            assert x.sum() == 0.0 and led[3] == 1.0


def test_pure_absorption_decay():
    mu_a, s_mm = 0.7, 0.1
    prob = _problem((16, 16, 16), [(0.0, mu_a, 0.9, 1.4)], s_mm=s_mm)
    A, _ = fcc.assemble(prob)
    st = fcc.site_index(prob.shape, (2, 2, 2)) * 12 + 11       # direction 11: (0, 1, 1) / sqrt 2
    for t in (1, 4, 9):
        x, _ = fcc.run(A, t, [st], [1.0], [1.0])
        assert x.sum() == pytest.approx(math.exp(-mu_a * s_mm * (t - 1)), rel=1e-14)
        assert x.min() >= 0.0


def test_ledger_closes_with_two_media():
    shape = (8, 6, 6)
    rng = np.random.default_rng(11)
    prob = _problem(shape, [(10.0, 0.02, 0.9, 1.4), (4.0, 0.3, 0.6, 1.4)],
                    medium=rng.integers(0, 2, size=8 * 6 * 6 // 2).astype(np.uint8))
    A, ex = fcc.assemble(prob)
    ab = fcc.absorb_fraction(prob)
    # every column: inside + exit + absorbed = 1 (Eq. 24 with open edges)
    assert np.allclose(np.asarray(A.sum(axis=0)).ravel() + ex + ab, 1.0, rtol=0, atol=1e-14)
    states = rng.integers(0, A.shape[0], size=5)
    weights = rng.random(5)
    prof = np.array([0.2, 0.5, 0.3])
    x, led = fcc.run(A, 30, states, weights, prof, t0=1, absorb=ab, exit_frac=ex)
    assert x.min() >= 0.0
    assert led[0] + led[2] + led[3] == pytest.approx(led[1], rel=1e-13)
    assert led[1] == pytest.approx(weights.sum(), rel=1e-14)


def _dense_transcription(shape, s_mm, medium_params):
    """Loop-literal A of Eq. 23 on the FCC box: for every source site and
    direction, every site of the box is tested directly against the point B
    (Eq. 18) and each segment A_m B (Eq. 19) in absolute coordinates."""
    nx, ny, nz = shape
    sites = [(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx) if (i + j + k) % 2 == 0]
    dirs = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dx != 0) + (dy != 0) + (dz != 0) == 2:
                    dirs.append((dx / S2, dy / S2, dz / S2))
    s = S2
    n_st = len(sites) * 12
    A = np.zeros((n_st, n_st))

    def dist_point(p, q):
        return math.sqrt(sum((p[c] - q[c]) ** 2 for c in range(3)))

    def dist_segment(p, a, b):
        d = [b[c] - a[c] for c in range(3)]
        dd = sum(v * v for v in d)
        if dd == 0.0:
            return dist_point(p, b)
        t = sum((p[c] - a[c]) * d[c] for c in range(3)) / dd
        t = min(1.0, max(0.0, t))
        return dist_point(p, [a[c] + t * d[c] for c in range(3)])

    for si, X in enumerate(sites):
        mu_s, mu_a, g = medium_params(si)
        L = s                                          # one refractive index: L = s
        Lmm = s_mm
        p_un = math.exp(-mu_s * Lmm) * math.exp(-mu_a * Lmm)
        p_sc = (1.0 - math.exp(-mu_s * Lmm)) * math.exp(-mu_a * Lmm)
        for n in range(12):
            hg = []
            for m in range(12):
                mu = sum(dirs[n][c] * dirs[m][c] for c in range(3))
                hg.append((1 - g * g) / (1 + g * g - 2 * g * mu) ** 1.5)
            hs = sum(hg)
            B = [X[c] + L * dirs[n][c] for c in range(3)]
            for m in range(12):
                Am = [X[c] + L * dirs[m][c] for c in range(3)]
                for kind in ("un", "sc"):
                    if kind == "un" and m != n:
                        continue
                    share = p_un if kind == "un" else p_sc * hg[m] / hs
                    # all lattice points near the segment, inside the box or not
                    lo = [int(math.floor(min(Am[c], B[c]) - s)) for c in range(3)]
                    hi = [int(math.ceil(max(Am[c], B[c]) + s)) for c in range(3)]
                    pts, ws = [], []
                    for k in range(lo[2], hi[2] + 1):
                        for j in range(lo[1], hi[1] + 1):
                            for i in range(lo[0], hi[0] + 1):
                                if (i + j + k) % 2:
                                    continue
                                d = dist_point((i, j, k), B) if kind == "un" else dist_segment((i, j, k), Am, B)
                                if d * d < s * s * (1 - 1e-9):
                                    pts.append((i, j, k))
                                    ws.append(s - d)
                    tot = sum(ws)
                    for p, w in zip(pts, ws):
                        if 0 <= p[0] < nx and 0 <= p[1] < ny and 0 <= p[2] < nz:
                            ti = ((p[2] * ny + p[1]) * nx + p[0]) // 2
                            A[ti * 12 + m, si * 12 + n] += share * w / tot
    return A


def test_dense_matrix_powers_against_transcription():
    shape, s_mm = (4, 4, 4), 0.1
    media = [(9.0, 0.05, 0.8, 1.4), (2.0, 0.4, 0.3, 1.4)]
    medium = np.array([(i * 7) % 3 == 0 for i in range(32)], dtype=np.uint8)
    prob = _problem(shape, media, medium=medium, s_mm=s_mm)
    A, _ = fcc.assemble(prob)
    D = _dense_transcription(shape, s_mm, lambda si: media[medium[si]][:3])
    assert np.allclose(A.toarray(), D, rtol=1e-13, atol=1e-16)
    # x(T) = sum_t A^(T-1-t) s(t) by dense powers vs the oracle's stepping
    src = [5, 100, 301]
    w = [1.0, 0.5, 2.0]
    prof = np.array([1.0, 0.25])
    T = 7
    s_vec = np.zeros(A.shape[0])
    for st, ww in zip(src, w):
        s_vec[st] += ww
    want = np.zeros(A.shape[0])
    for t in range(T):
        if t < len(prof):
            want += np.linalg.matrix_power(D, T - 1 - t) @ (s_vec * prof[t])
    x, _ = fcc.run(A, T, src, w, prof)
    assert np.allclose(x, want, rtol=1e-12, atol=1e-15)


def test_refractive_index_must_be_common():
    prob = _problem((4, 4, 4), [(1.0, 0.1, 0.5, 1.4), (1.0, 0.1, 0.5, 1.5)])
    with pytest.raises(ValueError):
        fcc.assemble(prob)


def _spread_unnormalised(Xf, dist, s):
    keep = dist * dist < s * s * fcc.MARGIN
    return keep, np.where(keep, s - dist, 0.0)


def _segment_to_source(X, A, B):
    # mistake: the segment runs from A_m to the source centre instead of B
    return fcc.__dict__["_segment_distance_orig"](X, A, np.zeros(3))


@pytest.mark.parametrize("plant", ["non_strict", "unnormalised", "segment_end"])
def test_planted_mistakes_are_caught(monkeypatch, plant):
    """Each plausible mistake in the FCC oracle fails at least one pin."""
    if plant == "non_strict":
        monkeypatch.setattr(fcc, "MARGIN", 1.0 + 1e-9)
    elif plant == "unnormalised":
        monkeypatch.setattr(fcc, "_spread", _spread_unnormalised)
    else:
        monkeypatch.setitem(fcc.__dict__, "_segment_distance_orig", fcc._segment_distance)
        monkeypatch.setattr(fcc, "_segment_distance", _segment_to_source)
    pins = [test_unscattered_lattice_direction_lands_on_one_neighbour,
            test_opposite_direction_segment_closed_form,
            lambda: test_column_sums_eq24(10.0, 0.01, 0.9)]
    failed = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1


def test_any_direction_set_keeps_eq24_column_sums():
    """The paper's own direction set (Lebedev points) is not carried here;
    the oracle's stencil takes any unit vectors.  With 26 directions that do
    not point at lattice sites, every source direction still sends out
    exactly e^{-mu_a L} (Eq. 24) and g = 0 spreads the scattered share
    evenly over the set."""
    v = np.array([(x, y, z) for z in (-1, 0, 1) for y in (-1, 0, 1) for x in (-1, 0, 1)
                  if (x, y, z) != (0, 0, 0)], dtype=np.float64)
    dirs = v / np.linalg.norm(v, axis=1, keepdims=True)
    mu_s, mu_a, s_mm = 6.0, 0.2, 0.1
    W = fcc.stencil(mu_s, mu_a, 0.0, 1.0, s_mm, dirs)
    tot = np.zeros(26)
    into = np.zeros((26, 26))
    for (n, _o, m), val in W.items():
        tot[n] += val
        into[n, m] += val
    assert np.allclose(tot, math.exp(-mu_a * s_mm), rtol=1e-14, atol=0)
    sc = (1.0 - math.exp(-mu_s * s_mm)) * math.exp(-mu_a * s_mm) / 26.0
    un = math.exp(-mu_s * s_mm) * math.exp(-mu_a * s_mm)
    assert np.allclose(into, sc + np.eye(26) * un, rtol=1e-13, atol=0)
