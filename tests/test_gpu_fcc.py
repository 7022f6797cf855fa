"""The Eq. 26 step on the close-packed (FCC) partition of Section 3, assembled
and run on the device (drts_fcc_assemble ... drts_fcc_step_n), against the
FP64 numpy oracle (oracle/fcc.py):
  * the device-assembled matrix read back row by row: row pointers and
    columns bit-exact, values to FP64 rounding (FP64) or the FP32 rounding
    of the oracle's value (FP32), on four boxes including two media, a
    two-site-wide box and a scattering-free medium;
  * multi-step states with a point source and a time profile (run lengths
    that leave part of the mass inside the open box): relative L1 <= 1e-12
    (FP64) and <= 1e-5 (FP32), including a box of 20,480 sites;
  * rejected inputs."""
import numpy as np
import pytest

from oracle import fcc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_08536_gb300 import build, drts
    build.build()
    drts.load()
    return drts


def _cases():
    rng = np.random.default_rng(5)
    return [
        ("homogeneous_8x6x6", (8, 6, 6), 0.1, [(10.0, 0.01, 0.9, 1.4)], None),
        ("two_media_10x8x6", (10, 8, 6), 0.08, [(10.0, 0.02, 0.9, 1.4), (4.0, 0.3, 0.6, 1.4)],
         rng.integers(0, 2, size=10 * 8 * 6 // 2)),
        ("thin_2x3x4", (2, 3, 4), 0.1, [(3.0, 0.1, 0.0, 1.33)], None),
        ("ballistic_6x6x6", (6, 6, 6), 0.1, [(0.0, 0.05, 0.5, 1.4)], None),
    ]


def _medium(shape, medium):
    n_sites = shape[0] * shape[1] * shape[2] // 2
    return np.zeros(n_sites, np.uint8) if medium is None else np.asarray(medium, np.uint8)


def rel_l1(a, b):
    return np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name,shape,s_mm,media,medium", _cases(), ids=[c[0] for c in _cases()])
def test_device_matrix_matches_oracle(gpu, name, shape, s_mm, media, medium, precision):
    medium = _medium(shape, medium)
    A, _ = fcc.assemble(fcc.FccProblem(shape, s_mm, media, medium))
    prec = gpu.FP64 if precision == "fp64" else gpu.FP32
    with gpu.FccContext(shape, s_mm, media, medium, precision=prec) as ctx:
        rp, col, val = ctx.read_rows()
        info = ctx.info()
        # a row range in the middle
        r0, r1 = 5 * 12 + 3, 9 * 12 + 7
        rp2, col2, _ = ctx.read_rows(r0, r1)
    assert np.array_equal(rp, A.indptr), name
    assert np.array_equal(col, A.indices), name
    assert info.nnz == A.nnz
    if precision == "fp64":
        assert np.allclose(val, A.data, rtol=1e-13, atol=0), name
    else:
        ref = A.data.astype(np.float32).astype(np.float64)
        ulp = np.spacing(np.abs(A.data).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(val - ref) <= ulp), name
    assert np.array_equal(rp2, A.indptr[r0:r1 + 1] - A.indptr[r0])
    assert np.array_equal(col2, A.indices[A.indptr[r0]:A.indptr[r1]])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("name,shape,s_mm,media,medium,steps", [
    ("homogeneous_8x6x6", (8, 6, 6), 0.1, [(10.0, 0.01, 0.9, 1.4)], None, 14),
    ("two_media_10x8x6", (10, 8, 6), 0.08, [(10.0, 0.02, 0.9, 1.4), (4.0, 0.3, 0.6, 1.4)], "random", 16),
    ("box_40x32x32", (40, 32, 32), 0.1, [(8.0, 0.02, 0.85, 1.4)], None, 40),
])
def test_device_steps_match_oracle(gpu, name, shape, s_mm, media, medium, steps, precision, tol):
    n_sites = shape[0] * shape[1] * shape[2] // 2
    if medium == "random":
        medium = np.random.default_rng(7).integers(0, len(media), size=n_sites)
    medium = _medium(shape, medium)
    A, _ = fcc.assemble(fcc.FccProblem(shape, s_mm, media, medium))
    nx, ny, nz = shape
    centre = fcc.site_index(shape, (nx // 2 if (nx // 2 + ny // 2 + nz // 2) % 2 == 0 else nx // 2 + 1,
                                    ny // 2, nz // 2))
    states = [centre * 12 + 3, centre * 12 + 8]
    weights = [0.75, 0.25]
    profile = np.exp(-0.5 * ((np.arange(12) - 5.0) / 2.0) ** 2)
    x_ref, _ = fcc.run(A, steps, states, weights, profile, t0=2)
    prec = gpu.FP64 if precision == "fp64" else gpu.FP32
    with gpu.FccContext(shape, s_mm, media, medium, precision=prec) as ctx:
        ctx.set_source(states, weights, profile, t0=2)
        ctx.step_n(steps // 2)
        ctx.step_n(steps - steps // 2)
        x = ctx.read_state()
        assert ctx.info().t == steps
    e = rel_l1(x, x_ref)
    print(f"close-packed {name} {precision} rel L1 after {steps} steps: {e:.3e}")
    assert x_ref.sum() > 0.01                 # mass is still in the box (the edges are open)
    assert e <= tol, (name, e)


def test_device_rejects_bad_input(gpu):
    med = [(10.0, 0.01, 0.9, 1.4)]
    with pytest.raises(gpu.DrtsError, match="nx must be even"):
        gpu.FccContext((5, 4, 4), 0.1, med, np.zeros(40, np.uint8))
    with pytest.raises(gpu.DrtsError, match="supports DRTS_FP64 and DRTS_FP32"):
        gpu.FccContext((4, 4, 4), 0.1, med, np.zeros(32, np.uint8), precision=gpu.FP16_ROWSCALE)
    with gpu.FccContext((4, 4, 4), 0.1, med, np.zeros(32, np.uint8)) as ctx:
        with pytest.raises(gpu.DrtsError, match="source state out of range"):
            ctx.set_source([32 * 12], [1.0], [1.0])
        with pytest.raises(gpu.DrtsError, match="repeated source state"):
            ctx.set_source([5, 5], [1.0, 1.0], [1.0])
        with pytest.raises(gpu.DrtsError, match="capacity"):
            ctx.read_rows(0, 24, cap=3)
