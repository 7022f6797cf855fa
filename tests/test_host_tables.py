"""The product's host-built tables (drts_host_tables: no device needed)
against the FP64 oracle on CPU: the stencil W_k[n][o][m] of Eq. 18-21 for
every medium, the exit fractions by face mask against the oracle's per-state
column functionals (Section 4.2, Eq. 27), and the FP16 row scales; with the
kernel's directions weighted alike and by their quadrature shares."""
import numpy as np
import pytest

from paper_1611_08536_gb300 import drts, inputs as I


def _problems():
    p1, _ = I.fresnel_cube(8, precision=I.FP64)
    p2, _ = I.three_layers(12, precision=I.FP32)
    p3, _ = I.inclusions(10, n_rhs=1, seed=2, precision=I.FP16_ROWSCALE, n_spheres=2)
    p3.boundary = I.OPEN
    p4, _ = I.ellipsoids(13, n_ell=4, seed=7, precision=I.FP32)      # media of differing n
    mov = np.zeros((7, 6, 5), np.uint8)
    mov[:, 3:, :] = 1
    p5 = I.Problem((5, 6, 7), 0.05, [(3.0, 0.2, 0.8, 1.33), (9.0, 0.02, 0.9, 1.5)], mov, 1.0,
                   I.MIRROR, I.FP64, 1, I.FACE_MX, 3, 2, "ragged_mirror")
    # the kernel weighting each direction by its quadrature share (R7 variant)
    q2, _ = I.three_layers(12, precision=I.FP32)
    q2.direction_weights = I.HG_QUADRATURE
    q5 = I.Problem((5, 6, 7), 0.05, [(3.0, 0.2, 0.8, 1.33), (9.0, 0.02, 0.9, 1.5)], mov, 1.0,
                   I.FRESNEL, I.FP16_ROWSCALE, 1, I.FACE_MX, 3, 2, "ragged_quadrature",
                   direction_weights=I.HG_QUADRATURE)
    return [("fresnel8", p1), ("layers12", p2), ("inclusions10_open_fp16", p3),
            ("ellipsoids13", p4), ("ragged_mirror", p5), ("layers12_quadrature", q2),
            ("ragged_quadrature_fp16", q5)]


@pytest.fixture(scope="module")
def lib():
    from paper_1611_08536_gb300 import build
    build.build()
    return drts.load()


@pytest.mark.parametrize("name,prob", _problems(), ids=[c[0] for c in _problems()])
def test_stencil_matches_oracle(lib, oracle_mod, name, prob):
    for k in range(len(prob.media)):
        W, _, _, _ = drts.host_tables(prob, k)
        Wo = oracle_mod.raw_stencil(prob, k)
        assert np.array_equal(W > 0.0, Wo > 0.0), (name, k)
        assert np.allclose(W, Wo, rtol=1e-14, atol=0), (name, k)


def _face_mask(shape):
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def b(c, n):
        return np.where(c == 0, 0, np.where(c == n - 1, 2, 1))
    return (b(z, nz) * 9 + b(y, ny) * 3 + b(x, nx)).ravel()


@pytest.mark.parametrize("name,prob", _problems(), ids=[c[0] for c in _problems()])
def test_exit_tables_match_oracle_column_functionals(lib, oracle_mod, name, prob):
    _, ex_o, ed_o, _ = oracle_mod.column_info(prob)
    mask = _face_mask(prob.shape)
    med = np.asarray(prob.medium_of_voxel).ravel()
    ex = np.empty_like(ex_o)
    ed = np.empty_like(ed_o)
    for k in range(len(prob.media)):
        _, ex_k, ed_k, _ = drts.host_tables(prob, k)
        sel = np.flatnonzero(med == k)
        ex.reshape(-1, 26)[sel] = ex_k[mask[sel]]
        ed.reshape(-1, 26)[sel] = ed_k[mask[sel]]
    assert np.allclose(ex, ex_o, rtol=1e-12, atol=1e-300), name
    assert np.allclose(ed, ed_o, rtol=1e-12, atol=1e-300), name


@pytest.mark.parametrize("name,prob", _problems(), ids=[c[0] for c in _problems()])
def test_fp16_row_scales(lib, name, prob):
    tabs = [drts.host_tables(prob, k) for k in range(len(prob.media))]
    sc = tabs[0][3]
    if prob.precision != I.FP16_ROWSCALE:
        assert np.all(sc == 1.0)
        return
    mant, _ = np.frexp(sc.astype(np.float64))
    assert np.all(mant == 0.5)                                  # powers of two
    wmax = np.max([t[0].max(axis=(0, 1)) for t in tabs], axis=0)   # per row direction m
    r = wmax / sc
    assert np.all((r > 2.0 ** 13) & (r <= 2.0 ** 14))


def test_bad_medium_is_rejected(lib):
    prob, _ = I.fresnel_cube(4, precision=I.FP32)
    with pytest.raises(drts.DrtsError) as e:
        drts.host_tables(prob, 1)
    assert e.value.status == drts.EINVAL
    assert "medium out of range" in str(e.value)


def test_quadrature_weighting_changes_the_kernel(lib):
    """The option is not inert: with g = 0 the equal kernel sends 1/26 of the
    scattered mass to every direction, the quadrature kernel 1/21, 4/105 and
    9/280 to axis, face-diagonal and body-diagonal directions."""
    prob = I.Problem((4, 4, 4), 0.1, [(5.0, 0.0, 0.0, 1.0)], np.zeros((4, 4, 4), np.uint8), 1.0,
                     I.MIRROR, I.FP64, 1, I.FACE_PZ, 2, 2, "g0")
    We, _, _, _ = drts.host_tables(prob, 0)
    prob.direction_weights = I.HG_QUADRATURE
    Wq, _, _, _ = drts.host_tables(prob, 0)
    unsc = np.exp(-0.5)
    n = I.direction_index(0, 0, 1)
    for W, expect in ((We, lambda m: 1.0 / 26.0),
                      (Wq, lambda m: {1: 1 / 21, 2: 4 / 105, 3: 9 / 280}[int(np.count_nonzero(I.direction_vector(m)))])):
        share = W[n].sum(axis=0)
        share[n] -= unsc
        for m in range(26):
            assert share[m] == pytest.approx(expect(m) * (1.0 - unsc), rel=1e-13)


def test_bad_direction_weights_rejected(lib):
    prob, _ = I.fresnel_cube(4, precision=I.FP32)
    prob.direction_weights = 2
    with pytest.raises(drts.DrtsError) as e:
        drts.host_tables(prob, 0)
    assert e.value.status == drts.EINVAL
