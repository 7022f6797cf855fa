"""The product's host-built two-step interface entries (drts_two_step_tables:
no device needed) against the FP64 oracle's (Section 4.2, planar interface
crossed in two parts) on CPU: which directions cross within the step, the
entries scattered before the plane (folded like the stencil) and the entries
reflected or refracted at it (folded at the grid edge only), on layered
problems with small and large index contrasts, a scattering-free layer, an
isotropic layer and a one-voxel layer between two others."""
import numpy as np
import pytest

from paper_1611_08536_gb300 import drts, inputs as I


def _layers(nz_of, media, name, shape=(6, 5, None), boundary=I.FRESNEL, precision=I.FP64):
    nz = len(nz_of)
    mov = np.empty((nz, shape[1], shape[0]), np.uint8)
    for z, k in enumerate(nz_of):
        mov[z] = k
    return I.Problem((shape[0], shape[1], nz), 0.1, media, mov, 1.0, boundary, precision, 1,
                     I.FACE_PZ, 2, 2, name, interface=I.INTERFACE_TWO_STEP)


def _problems():
    p1, _ = I.three_layers(12, precision=I.FP32)
    p1.interface = I.INTERFACE_TWO_STEP
    p2 = _layers([0, 0, 0, 1, 1, 1], [(10.0, 0.05, 0.9, 1.0), (10.0, 0.05, 0.9, 1.5)], "contrast_1_1.5")
    p3 = _layers([0, 0, 1, 1, 1], [(0.0, 0.02, 0.5, 1.33), (6.0, 0.1, 0.0, 1.4)], "ballistic_isotropic",
                 boundary=I.OPEN)
    p4 = _layers([0, 0, 1, 2, 2], [(8.0, 0.01, 0.8, 1.4), (12.0, 0.2, 0.7, 1.5), (5.0, 0.05, 0.95, 1.3)],
                 "thin_middle", boundary=I.MIRROR)
    p5 = _layers([0, 0, 0, 1, 1, 1], [(10.0, 0.05, 0.9, 1.0), (10.0, 0.05, 0.9, 1.5)], "contrast_quadrature")
    p5.direction_weights = I.HG_QUADRATURE      # the refracted piece's kernel weighted too
    return [("layers12", p1), ("contrast", p2), ("ballistic_isotropic", p3), ("thin_middle", p4),
            ("contrast_quadrature", p5)]


def _pairs(prob):
    mov = np.asarray(prob.medium_of_voxel)
    kz = [int(mov[z].ravel()[0]) for z in range(mov.shape[0])]
    out = set()
    for a, b in zip(kz[:-1], kz[1:]):
        if prob.media[a][3] != prob.media[b][3]:
            out.add((a, b))
            out.add((b, a))
    return sorted(out)


@pytest.fixture(scope="module")
def lib():
    from paper_1611_08536_gb300 import build
    build.build()
    return drts.load()


@pytest.mark.parametrize("name,prob", _problems(), ids=[c[0] for c in _problems()])
def test_two_step_entries_match_oracle(lib, oracle_mod, name, prob):
    pairs = _pairs(prob)
    assert pairs, name
    for k1, k2 in pairs:
        cross, fold, edge = drts.two_step_tables(prob, k1, k2)
        S1, S0, act = oracle_mod.two_step_stencil(prob, k1, k2)
        assert np.array_equal(cross, act.astype(np.uint8)), (name, k1, k2)
        assert cross.any(), (name, k1, k2)          # the axis direction always crosses
        for got, ref in ((fold, S1), (edge, S0)):
            assert np.array_equal(got > 0.0, ref > 0.0), (name, k1, k2)
            assert np.allclose(got, ref, rtol=1e-13, atol=0), (name, k1, k2)
        # directions that do not cross carry no two-step entries
        off = cross == 0
        assert not fold[off].any() and not edge[off].any()


def test_contrast_crossing_directions(lib, oracle_mod):
    """From the index-1.5 side only the axis directions (|S_z| = 1) reach the
    plane within the step (path 1/1.5 of a voxel; tc = 0.75), while from the
    index-1.0 side every direction with S_z != 0 does."""
    prob = _problems()[1][1]
    cross_hi, _, _ = drts.two_step_tables(prob, 1, 0)
    cross_lo, _, _ = drts.two_step_tables(prob, 0, 1)
    dz = np.array([I.direction_vector(d)[2] for d in range(26)])
    axis = np.array([np.count_nonzero(I.direction_vector(d)) == 1 for d in range(26)])
    assert np.array_equal(cross_hi.astype(bool), (dz != 0) & axis)
    assert np.array_equal(cross_lo.astype(bool), dz != 0)


def test_two_step_requests_rejected(lib):
    prob = _problems()[1][1]
    with pytest.raises(drts.DrtsError, match="do not meet"):
        drts.two_step_tables(prob, 0, 0)
    p = _problems()[1][1]
    p.interface = I.INTERFACE_FIRST_ORDER
    with pytest.raises(drts.DrtsError, match="not DRTS_INTERFACE_TWO_STEP"):
        drts.two_step_tables(p, 0, 1)
    # two-step interfaces need one medium per z layer
    q = _problems()[1][1]
    mov = np.array(q.medium_of_voxel)
    mov[2, 0, 0] = 1
    q.medium_of_voxel = mov
    with pytest.raises(drts.DrtsError, match="one medium per z layer"):
        drts.two_step_tables(q, 0, 1)
