"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Assembly: row pointers and column indices bit-exact, values within the
rounding of the stored precision.  Time step: relative L1 of the state
within the per-precision tolerance (FP64 1e-12; FP32 1e-5 per 1000 steps;
FP16 row-scaled 1e-4 or the measured figure stated in the test).
"""

import numpy as np
import pytest

from paper_1611_08536_gb300 import inputs as I

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


def rel_l1(a, b):
    return np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300)


def _val_tol(precision):
    # FP32 plain-row values use column-preserving rounding: within one ulp
    return {I.FP64: 1e-13, I.FP32: 2.0 ** -23 * 1.01, I.FP16_ROWSCALE: 2.0 ** -11}[precision]


def check_rows(ctx, csr, precision):
    r0, r1 = csr.row0, csr.row0 + csr.n_rows
    rp, col, val = ctx.export_rows(r0, r1, cap=csr.nnz + 16)
    assert np.array_equal(rp, csr.row_ptr)
    assert np.array_equal(col, csr.col)
    if precision == I.FP16_ROWSCALE:
        # FP16 times a power-of-two row scale, dithered rounding to a neighbour:
        # within one FP16 ulp of the value (plus the subnormal floor)
        rowmax = np.maximum.reduceat(csr.val, csr.row_ptr[:-1]) if csr.nnz else np.zeros(0)
        rm = np.repeat(rowmax, np.diff(csr.row_ptr))
        assert np.all(np.abs(val - csr.val) <= np.abs(csr.val) * 2.0 ** -10 + rm * 1e-9)
    else:
        assert np.all(np.abs(val - csr.val) <= np.abs(csr.val) * _val_tol(precision) + 1e-300)


def small_cases():
    out = []
    p, _ = I.fresnel_cube(9, precision=I.FP64)
    out.append(("fresnel9_fp64", p))
    p, _ = I.three_layers(16, precision=I.FP32)
    out.append(("layers16_fp32", p))
    p, _ = I.inclusions(10, n_rhs=1, seed=2, precision=I.FP32, n_spheres=2)
    p.boundary = I.OPEN
    out.append(("inclusions10_open_fp32", p))
    p, _ = I.ellipsoids(13, n_ell=4, seed=7, precision=I.FP32)
    out.append(("ellipsoids13_fp32", p))
    mov = np.zeros((7, 6, 5), np.uint8)
    mov[:, 3:, :] = 1
    p = I.Problem((5, 6, 7), 0.05, [(3.0, 0.2, 0.8, 1.33), (9.0, 0.02, 0.9, 1.5)], mov, 1.0,
                  I.MIRROR, I.FP64, 1, I.FACE_MX, 3, 2, "ragged_mirror")
    out.append(("ragged_5x6x7_mirror_fp64", p))
    p = I.Problem((2, 2, 2), 0.1, [(5.0, 0.1, 0.5, 1.4)], np.zeros((2, 2, 2), np.uint8), 1.0,
                  I.FRESNEL, I.FP32, 1, I.FACE_PZ, 1, 1, "tiny")
    out.append(("min_2x2x2_fp32", p))
    p, _ = I.three_layers(12, precision=I.FP16_ROWSCALE)
    out.append(("layers12_fp16", p))
    # the HG kernel's directions weighted by their quadrature shares
    p, _ = I.three_layers(10, precision=I.FP64)
    p.direction_weights = I.HG_QUADRATURE
    out.append(("layers10_quadrature_fp64", p))
    p = I.Problem((5, 6, 7), 0.05, [(3.0, 0.2, 0.8, 1.33), (9.0, 0.02, 0.9, 1.5)], mov, 1.0,
                  I.FRESNEL, I.FP32, 1, I.FACE_MX, 3, 2, "ragged_quadrature",
                  direction_weights=I.HG_QUADRATURE)
    out.append(("ragged_5x6x7_quadrature_fp32", p))
    return out


@pytest.mark.parametrize("name,prob", small_cases(), ids=[c[0] for c in small_cases()])
def test_assembly_matches_oracle(gpu, oracle_mod, name, prob):
    csr = oracle_mod.assemble(prob)
    with gpu.Context(prob) as ctx:
        check_rows(ctx, csr, prob.precision)
        info = ctx.info()
        assert info.nnz == csr.nnz
        if prob.precision == I.FP16_ROWSCALE:
            # the largest values of a row are kept as two FP16 terms: a few
            # per row, at least the unscattered streaming entries
            assert csr.nnz < info.nnz_stored < csr.nnz * 1.05
        else:
            assert info.nnz_stored == csr.nnz
        # column functionals
        ab, ex, ed = ctx.column_info()
        ab_o, ex_o, ed_o, _ = oracle_mod.column_info(prob)
        assert np.allclose(ab, ab_o, rtol=1e-14, atol=0)
        assert np.allclose(ex, ex_o, rtol=1e-12, atol=1e-300)
        assert np.allclose(ed, ed_o, rtol=1e-12, atol=1e-300)


def _run_both(gpu, oracle_mod, prob, src, steps, x0=None):
    csr = oracle_mod.assemble(prob)
    xo, deto, ledo = oracle_mod.run(prob, csr, steps, src.as_tuple(), x0=x0)
    with gpu.Context(prob, max_steps=steps) as ctx:
        if x0 is not None:
            ctx.write_state(x0)
        ctx.set_source(0, src)
        ctx.step_n(steps)
        x = ctx.read_state()
        det, led = ctx.read_detectors()
    return (x, det, led), (xo, deto, ledo)


def test_quadrature_weighted_kernel_fp64_steps(gpu, oracle_mod):
    """A run with the quadrature-weighted HG kernel follows the oracle's
    (FP64, three layers, Fresnel edges, 60 steps)."""
    prob, src = I.three_layers(10, precision=I.FP64)
    prob.direction_weights = I.HG_QUADRATURE
    (x, det, led), (xo, deto, ledo) = _run_both(gpu, oracle_mod, prob, src, 60)
    assert rel_l1(x, xo) < 1e-12
    assert rel_l1(det, deto) < 1e-12
    assert np.allclose(led, ledo, rtol=1e-11)


def test_fresnel_cube16_fp64_300_steps(gpu, oracle_mod):
    """16^3 FP64 configuration, delta pulse, 300 steps."""
    prob, src = I.fresnel_cube(16, precision=I.FP64)
    (x, det, led), (xo, deto, ledo) = _run_both(gpu, oracle_mod, prob, src, 300)
    assert rel_l1(x, xo) < 1e-12
    assert rel_l1(det, deto) < 1e-12
    assert np.allclose(led, ledo, rtol=1e-11)
    assert x.min() >= 0.0


def test_layers_fp32_1000_steps(gpu, oracle_mod):
    """Three-layer FP32 configuration at 24^3 for 1000 steps (tolerance 1e-5 per 1000 steps)."""
    prob, src = I.three_layers(24, precision=I.FP32)
    (x, det, led), (xo, deto, ledo) = _run_both(gpu, oracle_mod, prob, src, 1000)
    e = rel_l1(x, xo)
    print(f"FP32 rel L1 after 1000 steps: {e:.3e}")
    assert e <= 1e-5
    assert rel_l1(det, deto) <= 1e-5
    assert led[0] + led[2] + led[3] == pytest.approx(led[1], rel=1e-5)


@pytest.mark.parametrize("name,prob", small_cases()[2:6], ids=[c[0] for c in small_cases()[2:6]])
def test_step_random_state(gpu, oracle_mod, name, prob):
    rng = np.random.default_rng(5)
    x0 = rng.random(prob.n_states)
    src = I.Source(np.array([3, prob.n_states - 1], np.int64), np.array([0.5, 2.0]), 1,
                   np.array([1.0, 0.25, 4.0]))
    steps = 25
    (x, det, led), (xo, deto, ledo) = _run_both(gpu, oracle_mod, prob, src, steps, x0=x0)
    tol = 1e-12 if prob.precision == I.FP64 else 1e-5
    assert rel_l1(x, xo) < tol
    if det.size:
        assert rel_l1(det, deto) < tol
    assert led[1] == pytest.approx(ledo[1], rel=1e-12)


def _fp16_error(gpu, oracle_mod, steps):
    prob, src = I.three_layers(16, precision=I.FP16_ROWSCALE)
    (x, det, led), (xo, deto, ledo) = _run_both(gpu, oracle_mod, prob, src, steps)
    assert x.min() >= 0.0
    return rel_l1(x, xo)


def test_fp16_rowscale_meets_1e4(gpu, oracle_mod):
    e = _fp16_error(gpu, oracle_mod, 200)
    print(f"FP16-rowscale rel L1 after 200 steps: {e:.3e}")
    assert e < 1e-4


def test_fp16_rowscale_measured_bound(gpu, oracle_mod):
    """The FP16 tier's error at 16^3 three layers (37 % edge voxels) after 200
    steps.  A CPU emulation of the stored values on the oracle's matrix gives
    7.5e-6 with the large values of each row kept as two FP16 terms and the
    rest rounded by the spatial dither; the dither alone gave 1.9e-4, the
    earlier shared column-preserving rounding of the interior stencil 6.5e-3,
    nearest everywhere 3.0e-2."""
    e = _fp16_error(gpu, oracle_mod, 200)
    print(f"FP16-rowscale rel L1 after 200 steps: {e:.3e}")
    assert e < 3e-5


def test_fp16_rowscale_inclusions_500_steps(gpu, oracle_mod):
    """FP16 tier on a 24^3 cube with absorbing inclusions, 500 steps (dither
    alone emulated 1.4e-4, the shared-stencil rounding 1.1e-2)."""
    prob, srcs = I.inclusions(24, n_rhs=1, seed=3, precision=I.FP16_ROWSCALE)
    (x, det, led), (xo, deto, ledo) = _run_both(gpu, oracle_mod, prob, srcs[0], 500)
    e = rel_l1(x, xo)
    print(f"FP16-rowscale inclusions 24^3 rel L1 after 500 steps: {e:.3e}")
    assert e < 1e-4
    assert rel_l1(det, deto) < 1e-4


def test_empty_source_and_zero_steps(gpu):
    prob, _ = I.fresnel_cube(6, precision=I.FP32)
    with gpu.Context(prob, max_steps=5) as ctx:
        ctx.inject_source(0, [], [], 0, [])
        ctx.step_n(0)
        ctx.step_n(5)
        assert np.all(ctx.read_state() == 0.0)
        det, led = ctx.read_detectors()
        assert np.all(det == 0.0) and np.all(led == 0.0)
        with pytest.raises(gpu.DrtsError):
            ctx.step_n(1)                      # beyond max_steps


def test_invalid_inputs_rejected(gpu):
    prob, _ = I.fresnel_cube(4, precision=I.FP32)
    bad = I.Problem((1, 4, 4), 0.1, [(1, 0, 0, 1.4)], np.zeros((4, 4, 1), np.uint8))
    with pytest.raises(gpu.DrtsError):
        gpu.Context(bad)
    with gpu.Context(prob, max_steps=2) as ctx:
        with pytest.raises(gpu.DrtsError):
            ctx.inject_source(0, [prob.n_states], [1.0], 0, [1.0])
        with pytest.raises(gpu.DrtsError):
            ctx.inject_source(1, [0], [1.0], 0, [1.0])


def test_run_host_matches_step_n(gpu):
    prob, src = I.three_layers(16, precision=I.FP32)
    steps = 30
    with gpu.Context(prob, max_steps=steps) as a:
        a.set_source(0, src)
        a.step_n(steps)
        xa = a.read_state()
        da, _ = a.read_detectors()
    scale = np.zeros((steps, 1))
    t0, prof = src.t0, src.profile
    for t in range(steps):
        if t0 <= t < t0 + prof.size:
            scale[t, 0] = prof[t - t0]
    with gpu.Context(prob, max_steps=steps) as b:
        b.inject_source(0, src.state, src.weight, 0, [])
        det = np.zeros((steps, 1, 256))
        b.run_host(scale, det)
        xb = b.read_state()
    assert rel_l1(xb, xa) < 1e-6
    assert rel_l1(det[:, 0, :], da) < 1e-6


@pytest.mark.parametrize("variant", list(range(15)))
@pytest.mark.parametrize("precision", [I.FP64, I.FP32, I.FP16_ROWSCALE])
def test_step_variants_agree(gpu, oracle_mod, variant, precision):
    """Every launch variant of the step computes the same step (32 x 14 x 14
    so the halo variants, which need whole 32-voxel x-runs, apply)."""
    prob, _ = I.three_layers(14, precision=precision)
    mov = np.repeat(np.asarray(prob.medium_of_voxel)[:, :, :1], 32, axis=2)
    prob = I.Problem((32, 14, 14), prob.voxel_mm, prob.media, mov, prob.n_outside,
                     prob.boundary, precision, 1, prob.det_face, 14, 14, "layers_32x14x14")
    rng = np.random.default_rng(9)
    x0 = rng.random(prob.n_states)
    src = I.Source(np.array([prob.state(7, 7, 0, 21)], np.int64), np.ones(1), 0, np.ones(4))
    csr = oracle_mod.assemble(prob)
    xo, _, ledo = oracle_mod.run(prob, csr, 6, src.as_tuple(), x0=x0)
    with gpu.Context(prob, max_steps=6) as ctx:
        try:
            ctx.set_launch(0, 0, 0, variant)
        except gpu.DrtsError as e:
            if "does not fit" in str(e):
                pytest.skip(f"variant {variant} stages do not fit in shared memory at this precision")
            raise
        ctx.write_state(x0)
        ctx.set_source(0, src)
        ctx.step_n(6)
        x = ctx.read_state()
    tol = {I.FP64: 1e-12, I.FP32: 1e-6, I.FP16_ROWSCALE: 2e-3}[precision]
    assert rel_l1(x, xo) < tol


@pytest.mark.parametrize("variant,threads", [(9, 256), (10, 256), (10, 96), (11, 256), (11, 128), (12, 256),
                                            (13, 96), (14, 256)])
def test_step_variants_ragged_grid(gpu, oracle_mod, variant, threads):
    """The register variants that take any grid (pipelined, two and four
    and eight warps per slice, 32-bit indices) on a 13 x 11 x 9 FP64 grid whose 32-voxel blocks wrap
    across x rows, with detector and ledger, including block shapes whose
    warp count is not a multiple of the warps per slice."""
    prob, _ = I.three_layers(9, precision=I.FP64)
    mov = np.repeat(np.repeat(np.asarray(prob.medium_of_voxel)[:, :1, :1], 11, axis=1), 13, axis=2)
    prob = I.Problem((13, 11, 9), prob.voxel_mm, prob.media, mov, prob.n_outside,
                     prob.boundary, I.FP64, 1, prob.det_face, 4, 3, "layers_13x11x9")
    rng = np.random.default_rng(21)
    x0 = rng.random(prob.n_states)
    src = I.Source(np.array([prob.state(6, 5, 0, 21)], np.int64), np.ones(1), 0, np.ones(3))
    csr = oracle_mod.assemble(prob)
    xo, deto, ledo = oracle_mod.run(prob, csr, 8, src.as_tuple(), x0=x0)
    with gpu.Context(prob, max_steps=8) as ctx:
        ctx.set_launch(0, threads, 0, variant)
        ctx.write_state(x0)
        ctx.set_source(0, src)
        ctx.step_n(8)
        x = ctx.read_state()
        det, led = ctx.read_detectors()
    assert rel_l1(x, xo) < 1e-12
    assert rel_l1(det, deto) < 1e-12
    assert np.allclose(led[1:], ledo[1:], rtol=1e-11)


def test_bounded_wait_times_out_and_recovers(gpu, oracle_mod):
    """A copy that is never issued makes the bulk-copy step's bounded wait run
    out: DRTS_ETIMEOUT is reported and the context stays usable."""
    prob, _ = I.three_layers(12, precision=I.FP32)
    rng = np.random.default_rng(3)
    x0 = rng.random(prob.n_states)
    csr = oracle_mod.assemble(prob)
    with gpu.Context(prob, max_steps=4) as ctx:
        ctx.set_launch(0, 0, 0, 3)
        ctx.set_fault(gpu.FAULT_SPIN_LIMIT, 2000)
        ctx.set_fault(gpu.FAULT_SKIP_COPY, 0)
        ctx.write_state(x0)
        ctx.step_n(1)
        with pytest.raises(gpu.DrtsError) as ei:
            ctx.read_state()
        assert ei.value.status == gpu.ETIMEOUT
        ctx.set_fault(gpu.FAULT_NONE)
        ctx.write_state(x0)
        ctx.step_n(1)
        x1 = ctx.read_state()
    assert rel_l1(x1, oracle_mod.spmv(csr, x0)) < 1e-6


def test_autotune_keeps_state_and_parity(gpu, oracle_mod):
    prob, src = I.three_layers(16, precision=I.FP32)
    csr = oracle_mod.assemble(prob)
    rng = np.random.default_rng(4)
    x0 = rng.random(prob.n_states)
    with gpu.Context(prob, max_steps=3) as ctx:
        ctx.write_state(x0)
        before = ctx.read_state()
        r = ctx.autotune(2)
        # 16^3: the halo variants (7, 8: whole 32-voxel x-runs only) do not apply
        assert 0 <= r["variant"] < 15 and r["variant"] not in (7, 8)
        assert r["candidates"] > 0 and r["ms_per_step"] > 0
        assert np.array_equal(ctx.read_state(), before)
        det, led = ctx.read_detectors()
        assert np.all(led[1:] == 0.0)              # trial steps leave the ledger alone
        ctx.step_n(1)
        x1 = ctx.read_state()
        r2 = ctx.autotune(2)                       # cached in-process
        assert r2["from_cache"] == 1 and r2["variant"] == r["variant"]
    assert rel_l1(x1, oracle_mod.spmv(csr, before)) < 1e-6


def test_persistent_fp64_300_steps(gpu, oracle_mod):
    """The persistent multi-step kernel on the 16^3 FP64 configuration."""
    prob, src = I.fresnel_cube(16, precision=I.FP64)
    csr = oracle_mod.assemble(prob)
    xo, deto, ledo = oracle_mod.run(prob, csr, 300, src.as_tuple())
    with gpu.Context(prob, max_steps=300) as ctx:
        ctx.set_step_mode(gpu.STEP_PERSISTENT)
        ctx.set_source(0, src)
        ctx.step_n(300)
        x = ctx.read_state()
        det, led = ctx.read_detectors()
    assert rel_l1(x, xo) < 1e-12
    assert rel_l1(det, deto) < 1e-12
    assert np.allclose(led, ledo, rtol=1e-11)


@pytest.mark.parametrize("variant,threads", [(10, 256), (10, 64), (11, 256), (11, 128), (14, 256)])
def test_persistent_split_slices(gpu, oracle_mod, variant, threads):
    """After a split launch variant (two, four or eight warps per slice) the
    persistent kernel splits its slices the same way."""
    prob, src = I.fresnel_cube(12, precision=I.FP64)
    csr = oracle_mod.assemble(prob)
    xo, deto, ledo = oracle_mod.run(prob, csr, 40, src.as_tuple())
    with gpu.Context(prob, max_steps=40) as ctx:
        ctx.set_launch(0, threads, 0, variant)
        ctx.set_step_mode(gpu.STEP_PERSISTENT)
        ctx.set_source(0, src)
        ctx.step_n(40)
        x = ctx.read_state()
        det, led = ctx.read_detectors()
    assert rel_l1(x, xo) < 1e-12
    assert rel_l1(det, deto) < 1e-12
    assert np.allclose(led, ledo, rtol=1e-11)


def test_persistent_mixed_with_launches(gpu, oracle_mod):
    prob, src = I.three_layers(16, precision=I.FP32)
    csr = oracle_mod.assemble(prob)
    rng = np.random.default_rng(2)
    x0 = rng.random(prob.n_states)
    xo, deto, _ = oracle_mod.run(prob, csr, 25, src.as_tuple(), x0=x0)
    with gpu.Context(prob, max_steps=25) as ctx:
        ctx.write_state(x0)
        ctx.set_source(0, src)
        ctx.set_step_mode(gpu.STEP_PERSISTENT)
        ctx.step_n(9)
        ctx.set_step_mode(gpu.STEP_LAUNCH)
        ctx.step_n(5)
        ctx.set_step_mode(gpu.STEP_PERSISTENT)
        ctx.step_n(11)
        x = ctx.read_state()
        det, _ = ctx.read_detectors()
    assert rel_l1(x, xo) < 1e-6
    assert rel_l1(det, deto) < 1e-6


def test_persistent_barrier_times_out_and_recovers(gpu, oracle_mod):
    """A block that never arrives at the grid barrier makes the other blocks'
    bounded waits run out: DRTS_ETIMEOUT, and the context stays usable."""
    prob, _ = I.three_layers(12, precision=I.FP32)
    csr = oracle_mod.assemble(prob)
    rng = np.random.default_rng(6)
    x0 = rng.random(prob.n_states)
    with gpu.Context(prob, max_steps=8) as ctx:
        ctx.set_step_mode(gpu.STEP_PERSISTENT)
        ctx.set_fault(gpu.FAULT_SPIN_LIMIT, 5000)
        ctx.set_fault(gpu.FAULT_SKIP_BARRIER, 0)
        ctx.write_state(x0)
        ctx.step_n(3)
        with pytest.raises(gpu.DrtsError) as ei:
            ctx.read_state()
        assert ei.value.status == gpu.ETIMEOUT
        ctx.set_fault(gpu.FAULT_NONE)
        ctx.write_state(x0)
        ctx.step_n(2)
        x2 = ctx.read_state()
    assert rel_l1(x2, oracle_mod.spmv(csr, oracle_mod.spmv(csr, x0))) < 1e-6


@pytest.mark.parametrize("precision", [I.FP32, I.FP64])
def test_checkpoint_resume_equals_uninterrupted(gpu, precision):
    prob, src = I.three_layers(16, precision=precision)
    with gpu.Context(prob, max_steps=40) as a:
        a.set_source(0, src)
        a.step_n(40)
        xa = a.read_state()
        da, la = a.read_detectors()
    with gpu.Context(prob, max_steps=40) as b:
        b.set_source(0, src)
        b.step_n(17)
        data = b.checkpoint()
    with gpu.Context(prob, max_steps=40) as c:
        c.set_source(0, src)
        c.restore(data)
        assert c.info().t == 17
        c.step_n(23)
        xc = c.read_state()
        dc, lc = c.read_detectors()
    assert np.array_equal(xa, xc)                 # the state is deterministic
    assert rel_l1(dc, da) < 1e-12
    assert np.allclose(lc, la, rtol=1e-12)
    with gpu.Context(prob, max_steps=40) as e:    # restore into a context that has stepped
        e.set_source(0, src)
        e.step_n(3)
        e.restore(data)
        assert e.info().t == 17
        e.step_n(23)
        assert np.array_equal(xa, e.read_state())
    other, _ = I.three_layers(12, precision=precision)
    with gpu.Context(other, max_steps=40) as d:
        with pytest.raises(gpu.DrtsError):
            d.restore(data)
