"""Pins of the oracle's Eq. 26/27 extensions: sparse detector rows (a point
detector reads chosen (voxel, direction) states), the sensor response of
Eq. 27 (impulse response over a time window) and the source column of a
population emitted during a step (Section 4.1 time partition of the source).

Each pin is a closed form, an exact invariant, a library routine on a special
case, or the oracle's own state read another way.
"""
import math

import numpy as np
import pytest

from paper_1611_08536_gb300 import inputs as I

D = I.direction_index


def _prob(n, media, boundary=I.MIRROR, mov=None, h=0.1, n_out=1.0, det=(I.FACE_PZ, 2, 2)):
    shape = (n, n, n) if isinstance(n, int) else n
    if mov is None:
        mov = np.zeros(shape[::-1], np.uint8)
    return I.Problem(shape, h, list(media), mov, n_out, boundary, I.FP64, 1,
                     det[0], det[1], det[2])


def _delta(prob, x, y, z, d, t0=0):
    return (np.array([prob.state(x, y, z, d)], np.int64), np.ones(1), t0, np.ones(1))


# --------------------------------------------------------------------------
# Eq. 27 with a general F: sparse detector rows


def test_point_rows_with_exit_weights_reproduce_face_detector(oracle_mod):
    """F = exit coefficient over each face patch (the definition of the face
    detector) gives the face detector's readout, bit for bit (same order)."""
    prob = _prob(6, [(8.0, 0.05, 0.8, 1.4)], boundary=I.FRESNEL, det=(I.FACE_PZ, 2, 3))
    csr = oracle_mod.assemble(prob)
    ab, ex, ed, patch = oracle_mod.column_info(prob)
    sel = np.flatnonzero((patch >= 0) & (ed > 0))
    point = (int(patch.max()) + 1, patch[sel], sel, ed[sel])
    src = _delta(prob, 3, 2, 0, D(0, 0, 1))
    x, det, led, pdet = oracle_mod.run(prob, csr, 30, src, point=point)
    assert det.any()
    assert np.array_equal(pdet, det)


def test_point_row_reads_the_state(oracle_mod):
    """A one-entry row (s, w) reads w * x_t[s]; x_t from separate runs of t steps."""
    prob = _prob(5, [(6.0, 0.1, 0.7, 1.3)], boundary=I.FRESNEL)
    csr = oracle_mod.assemble(prob)
    s = prob.state(2, 2, 2, D(0, 0, 1))
    s2 = prob.state(2, 3, 2, D(0, 1, 0))
    point = (2, np.array([0, 1, 1], np.int32), np.array([s, s2, s], np.int64),
             np.array([2.5, 1.0, -0.5]))
    src = _delta(prob, 2, 2, 0, D(0, 0, 1))
    T = 7
    _, _, _, pdet = oracle_mod.run(prob, csr, T, src, point=point)
    for t in range(1, T):
        xt, _, _ = oracle_mod.run(prob, csr, t, src)
        assert pdet[t, 0] == 2.5 * xt[s]
        assert pdet[t, 1] == pytest.approx(xt[s2] - 0.5 * xt[s], rel=1e-15, abs=1e-300)
    assert pdet[0].tolist() == [0.0, 0.0]


def test_point_rows_total_mass_closed_box(oracle_mod):
    """F = 1 on every state in a mirror box without absorption: the detector
    reads the conserved mass, 0 before the delta pulse and 1 after it."""
    prob = _prob(4, [(5.0, 0.0, 0.9, 1.0)], boundary=I.MIRROR)
    csr = oracle_mod.assemble(prob)
    n = prob.n_states
    point = (1, np.zeros(n, np.int32), np.arange(n, dtype=np.int64), np.ones(n))
    _, _, _, pdet = oracle_mod.run(prob, csr, 12, _delta(prob, 1, 2, 3, D(1, 0, -1), t0=2),
                                   point=point)
    assert pdet[:3, 0].tolist() == [0.0, 0.0, 0.0]
    np.testing.assert_allclose(pdet[3:, 0], 1.0, rtol=1e-13)


def test_point_rows_reject_bad_entries(oracle_mod):
    prob = _prob(3, [(1.0, 0.0, 0.0, 1.0)])
    csr = oracle_mod.assemble(prob)
    bad = (1, np.array([1], np.int32), np.array([0], np.int64), np.ones(1))
    with pytest.raises(RuntimeError):
        oracle_mod.run(prob, csr, 2, _delta(prob, 0, 0, 0, 0), point=bad)


# --------------------------------------------------------------------------
# Eq. 27: sensor impulse response over a window of +-w steps


def _series(T=40, n_det=3, seed=1):
    return np.random.default_rng(seed).random((T, n_det))


def test_sensor_delta_response_is_identity(oracle_mod):
    Dm = _series()
    assert np.array_equal(oracle_mod.sensor_response(Dm, 0, [1.0]), Dm)
    h = np.zeros(7)
    h[3] = 1.0
    assert np.array_equal(oracle_mod.sensor_response(Dm, 3, h), Dm)


def test_sensor_delayed_impulse_shifts(oracle_mod):
    """h = delta at lag +2: the sensor reports the photons of two steps earlier."""
    Dm = _series()
    h = np.zeros(7)
    h[3 + 2] = 1.0
    M = oracle_mod.sensor_response(Dm, 3, h)
    assert np.array_equal(M[2:], Dm[:-2])
    assert not M[:2].any()


def test_sensor_box_window_matches_library_convolution(oracle_mod):
    Dm = _series(T=33)
    M = oracle_mod.sensor_response(Dm, 2, np.ones(5))
    for d in range(Dm.shape[1]):
        np.testing.assert_allclose(M[:, d], np.convolve(Dm[:, d], np.ones(5), mode="same"),
                                   rtol=1e-14)


def test_sensor_asymmetric_kernel_matches_library_convolution(oracle_mod):
    """A causal exponential response, h[j + w] = exp(-j / 2) for lags j >= 0."""
    Dm = _series(T=50, seed=4)
    w = 6
    lags = np.arange(-w, w + 1)
    h = np.where(lags >= 0, np.exp(-lags / 2.0), 0.0)
    M = oracle_mod.sensor_response(Dm, w, h)
    for d in range(Dm.shape[1]):
        full = np.convolve(Dm[:, d], h)            # full[t + w] = sum_k D[k] h[t - k + w]
        np.testing.assert_allclose(M[:, d], full[w:w + Dm.shape[0]], rtol=1e-13)


def test_sensor_response_linear(oracle_mod):
    D1, D2 = _series(seed=2), _series(seed=3)
    h = np.random.default_rng(5).random(9)
    M = oracle_mod.sensor_response(3.0 * D1 - 0.5 * D2, 4, h)
    ref = 3.0 * oracle_mod.sensor_response(D1, 4, h) - 0.5 * oracle_mod.sensor_response(D2, 4, h)
    np.testing.assert_allclose(M, ref, rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------
# Section 4.1: source population emitted during a step travels frac * L


@pytest.mark.parametrize("frac", [0.25, 0.5, 0.8, 1.0])
def test_source_column_axis_closed_form(oracle_mod, frac):
    """No scattering, axis direction: the end point X + f h e_z lies between
    the source voxel (distance f h) and the next one ((1 - f) h); every other
    lattice point is at least h away, so Eq. 18 gives weights 1 - f and f,
    times the absorption survival exp(-mu_a f h)."""
    mu_a = 0.3
    prob = _prob(5, [(0.0, mu_a, 0.0, 1.0)], h=0.2)
    s = prob.state(2, 2, 2, D(0, 0, 1))
    st, w, ex = oracle_mod.source_column(prob, s, frac)
    surv = math.exp(-mu_a * frac * 0.2)
    if frac == 1.0:
        assert st.tolist() == [prob.state(2, 2, 3, D(0, 0, 1))]
        assert w[0] == pytest.approx(surv, rel=1e-15)
    else:
        assert st.tolist() == [s, prob.state(2, 2, 3, D(0, 0, 1))]
        np.testing.assert_allclose(w, [(1 - frac) * surv, frac * surv], rtol=1e-14)
    assert ex == 0.0


@pytest.mark.parametrize("frac", [0.3, 0.7])
@pytest.mark.parametrize("d", [(1, 0, 0), (1, 1, 0), (-1, 1, 1)])
def test_source_column_sum_is_absorption_survival(oracle_mod, frac, d):
    """Interior source, any scattering: the column sums to exp(-mu_a f L)
    (Eq. 24 for a partial path), whatever mu_s and g."""
    mu_a = 0.05
    prob = _prob(5, [(10.0, mu_a, 0.9, 1.4)], h=0.1)
    s = prob.state(2, 2, 2, D(*d))
    st, w, ex = oracle_mod.source_column(prob, s, frac)
    assert w.sum() == pytest.approx(math.exp(-mu_a * frac * 0.1), rel=1e-13)
    assert (w > 0).all() and ex == 0.0
    assert np.all(np.diff(st) > 0)


def test_source_column_short_path_is_dirac(oracle_mod):
    """As f -> 0 the population stays in its own state (the plain source term
    of Eq. 26)."""
    prob = _prob(4, [(10.0, 0.05, 0.9, 1.4)], h=0.1)
    s = prob.state(1, 2, 1, D(0, -1, 1))
    st, w, _ = oracle_mod.source_column(prob, s, 1e-12)
    k = list(st).index(s)
    assert w[k] == pytest.approx(1.0, abs=1e-10)
    assert np.delete(w, k).sum() < 1e-10


def test_source_column_full_step_equals_system_matrix_column(oracle_mod):
    """f = 1 is column (i, n) of A, including edge and interface folding."""
    mov = np.zeros((4, 4, 4), np.uint8)
    mov[2:] = 1
    prob = _prob(4, [(6.0, 0.02, 0.8, 1.4), (3.0, 0.05, 0.6, 1.5)], boundary=I.FRESNEL, mov=mov)
    csr = oracle_mod.assemble(prob)
    import scipy.sparse as sp
    A = sp.csr_matrix((csr.val, csr.col, csr.row_ptr), shape=(csr.n_rows, csr.n_rows)).tocsc()
    for (x, y, z, d) in [(0, 0, 0, D(1, 1, 1)), (1, 2, 1, D(0, 0, 1)), (3, 1, 2, D(1, 0, -1))]:
        s = prob.state(x, y, z, d)
        st, w, _ = oracle_mod.source_column(prob, s, 1.0)
        col = A[:, s]
        assert st.tolist() == col.indices.tolist()
        np.testing.assert_allclose(w, col.data, rtol=1e-14)


@pytest.mark.parametrize("frac", [0.2, 0.6, 1.0])
def test_source_column_mirror_conserves_mass_at_corner(oracle_mod, frac):
    prob = _prob(4, [(7.0, 0.0, 0.85, 1.3)], boundary=I.MIRROR)
    s = prob.state(0, 0, 0, D(-1, -1, -1))
    _, w, ex = oracle_mod.source_column(prob, s, frac)
    assert w.sum() == pytest.approx(1.0, rel=1e-13)
    assert ex == 0.0


def test_source_column_fresnel_edge_balance(oracle_mod):
    """At a Fresnel face the kept and the exiting mass add up to the
    absorption survival of the partial path."""
    mu_a, frac = 0.04, 0.5
    prob = _prob(4, [(9.0, mu_a, 0.9, 1.4)], boundary=I.FRESNEL, h=0.1)
    s = prob.state(0, 1, 2, D(-1, 0, 0))
    _, w, ex = oracle_mod.source_column(prob, s, frac)
    assert ex > 0
    assert w.sum() + ex == pytest.approx(math.exp(-mu_a * frac * 0.1), rel=1e-13)


def test_source_column_rejects_bad_input(oracle_mod):
    prob = _prob(3, [(1.0, 0.0, 0.0, 1.0)])
    for frac in (0.0, -0.1, 1.5):
        with pytest.raises(ValueError):
            oracle_mod.source_column(prob, 0, frac)
    with pytest.raises(ValueError):
        oracle_mod.source_column(prob, prob.n_states, 0.5)
