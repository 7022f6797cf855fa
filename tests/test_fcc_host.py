"""Host assembly of the close-packed (FCC) partition in the product
(drts_fcc_host_rows, C++) against the numpy oracle of Section 3: row
pointers and columns bit-exact, values to FP64 rounding.  No device."""
import numpy as np
import pytest

from oracle import fcc
from paper_1611_08536_gb300 import drts


def _cases():
    rng = np.random.default_rng(5)
    return [
        ("homogeneous_8x6x6", (8, 6, 6), 0.1, [(10.0, 0.01, 0.9, 1.4)], None),
        ("two_media_10x8x6", (10, 8, 6), 0.08, [(10.0, 0.02, 0.9, 1.4), (4.0, 0.3, 0.6, 1.4)],
         rng.integers(0, 2, size=10 * 8 * 6 // 2)),
        ("thin_2x3x4", (2, 3, 4), 0.1, [(3.0, 0.1, 0.0, 1.33)], None),
        ("ballistic_6x6x6", (6, 6, 6), 0.1, [(0.0, 0.05, 0.5, 1.4)], None),
    ]


@pytest.fixture(scope="module")
def lib():
    from paper_1611_08536_gb300 import build
    build.build()
    return drts.load()


@pytest.mark.parametrize("name,shape,s_mm,media,medium", _cases(), ids=[c[0] for c in _cases()])
def test_host_rows_match_oracle(lib, name, shape, s_mm, media, medium):
    n_sites = shape[0] * shape[1] * shape[2] // 2
    if medium is None:
        medium = np.zeros(n_sites, np.uint8)
    medium = np.asarray(medium, np.uint8)
    A, _ = fcc.assemble(fcc.FccProblem(shape, s_mm, media, medium))
    rp, col, val = drts.fcc_host_rows(shape, s_mm, media, medium)
    assert np.array_equal(rp, A.indptr), name
    assert np.array_equal(col, A.indices), name
    assert np.allclose(val, A.data, rtol=1e-13, atol=0), name
    # a row range in the middle
    r0, r1 = 5 * 12 + 3, 9 * 12 + 7
    rp2, col2, val2 = drts.fcc_host_rows(shape, s_mm, media, medium, r0, r1)
    assert np.array_equal(rp2, A.indptr[r0:r1 + 1] - A.indptr[r0])
    assert np.array_equal(col2, A.indices[A.indptr[r0]:A.indptr[r1]])


def test_host_rows_reject_bad_input(lib):
    med = [(10.0, 0.01, 0.9, 1.4)]
    with pytest.raises(drts.DrtsError, match="nx must be even"):
        drts.fcc_host_rows((5, 4, 4), 0.1, med, np.zeros(40, np.uint8))
    with pytest.raises(drts.DrtsError, match="one refractive index"):
        drts.fcc_host_rows((4, 4, 4), 0.1, med + [(1.0, 0.1, 0.5, 1.5)], np.zeros(32, np.uint8))
    with pytest.raises(drts.DrtsError, match="capacity"):
        drts.fcc_host_rows((4, 4, 4), 0.1, med, np.zeros(32, np.uint8), cap=10)
    with pytest.raises(drts.DrtsError, match="bad row range"):
        drts.fcc_host_rows((4, 4, 4), 0.1, med, np.zeros(32, np.uint8), 0, 32 * 12 + 1)
