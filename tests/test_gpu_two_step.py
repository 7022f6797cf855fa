"""Planar interfaces crossed in two steps (DRTS_INTERFACE_TWO_STEP, Section
4.2) on the device, through the C ABI, against the FP64 oracle with the same
option:
  * the device-assembled A: row pointers and columns bit-exact, values to the
    stored precision's rounding, on layered problems with small and large
    index contrasts, every edge treatment, a scattering-free layer, a
    one-voxel layer between two others, a ragged grid and the FP16 tier;
  * the per-state column functionals (absorbed and exiting mass, detector
    face share) of the step's ledger;
  * multi-step states, detector readouts and the ledger: FP64 single
    right-hand side, FP32 single and batched (CUDA cores and tensor cores);
  * the first-order and two-step matrices differ only in rows near an
    index change, and a non-layered medium map is rejected."""
import copy

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


def _layers(kz, media, name, shape=(7, 6), boundary=I.FRESNEL, precision=I.FP64, n_rhs=1,
            det_face=I.FACE_PZ):
    mov = np.empty((len(kz), shape[1], shape[0]), np.uint8)
    for z, k in enumerate(kz):
        mov[z] = k
    return I.Problem((shape[0], shape[1], len(kz)), 0.1, media, mov, 1.0, boundary, precision, n_rhs,
                     det_face, 2, 2, name, interface=I.INTERFACE_TWO_STEP)


def cases():
    p1, _ = I.three_layers(12, precision=I.FP32)
    p1.interface = I.INTERFACE_TWO_STEP
    p2 = _layers([0, 0, 0, 1, 1, 1, 1], [(10.0, 0.05, 0.9, 1.0), (10.0, 0.05, 0.9, 1.5)], "contrast_fp64")
    p3 = _layers([0, 0, 1, 1, 1, 1], [(0.0, 0.02, 0.5, 1.33), (6.0, 0.1, 0.0, 1.4)], "ballistic_open_fp64",
                 boundary=I.OPEN)
    p4 = _layers([0, 0, 1, 2, 2, 2], [(8.0, 0.01, 0.8, 1.4), (12.0, 0.2, 0.7, 1.5), (5.0, 0.05, 0.95, 1.3)],
                 "thin_middle_mirror_fp32", boundary=I.MIRROR, precision=I.FP32)
    p5 = _layers([1, 0, 0, 1, 1, 0, 0], [(9.0, 0.02, 0.9, 1.37), (14.0, 0.04, 0.85, 1.45)], "ragged_5x3_fp32",
                 shape=(5, 3), precision=I.FP32, det_face=I.FACE_MX)
    p6, _ = I.three_layers(12, precision=I.FP16_ROWSCALE)
    p6.interface = I.INTERFACE_TWO_STEP
    return [("layers12_fp32", p1), ("contrast_fp64", p2), ("ballistic_open_fp64", p3),
            ("thin_middle_mirror_fp32", p4), ("ragged_5x3_fp32", p5), ("layers12_fp16", p6)]


def check_rows(ctx, csr, precision):
    r0, r1 = csr.row0, csr.row0 + csr.n_rows
    rp, col, val = ctx.export_rows(r0, r1, cap=csr.nnz + 16)
    assert np.array_equal(rp, csr.row_ptr)
    assert np.array_equal(col, csr.col)
    if precision == I.FP16_ROWSCALE:
        rowmax = np.maximum.reduceat(csr.val, csr.row_ptr[:-1])
        rm = np.repeat(rowmax, np.diff(csr.row_ptr))
        assert np.all(np.abs(val - csr.val) <= np.abs(csr.val) * 2.0 ** -10 + rm * 1e-9)
    else:
        tol = 1e-13 if precision == I.FP64 else 2.0 ** -23 * 1.01
        assert np.all(np.abs(val - csr.val) <= np.abs(csr.val) * tol + 1e-300)


@pytest.mark.parametrize("name,prob", cases(), ids=[c[0] for c in cases()])
def test_two_step_assembly_matches_oracle(gpu, oracle_mod, name, prob):
    csr = oracle_mod.assemble(prob)
    with gpu.Context(prob) as ctx:
        check_rows(ctx, csr, prob.precision)


@pytest.mark.parametrize("name,prob", cases()[:5], ids=[c[0] for c in cases()[:5]])
def test_two_step_column_functionals_match_oracle(gpu, oracle_mod, name, prob):
    ab_o, ex_o, ed_o, _ = oracle_mod.column_info(prob)
    with gpu.Context(prob) as ctx:
        ab, ex, ed = ctx.column_info()
    assert np.allclose(ab, ab_o, rtol=1e-12, atol=1e-15), name
    assert np.allclose(ex, ex_o, rtol=1e-12, atol=1e-15), name
    assert np.allclose(ed, ed_o, rtol=1e-12, atol=1e-15), name


def test_two_step_changes_only_rows_near_an_interface(gpu, oracle_mod):
    """The two-step rows differ from the first-order ones only within two z
    layers of an index change; every other row is identical."""
    prob = cases()[1][1]
    p1 = copy.copy(prob)
    p1.interface = I.INTERFACE_FIRST_ORDER
    with gpu.Context(prob) as c2, gpu.Context(p1) as c1:
        rp2, col2, val2 = c2.export_rows(0, prob.n_states)
        rp1, col1, val1 = c1.export_rows(0, prob.n_states)
    nx, ny, nz = prob.shape
    rows_per_layer = nx * ny * 26
    differ = set()
    for r in range(prob.n_states):
        a = (col1[rp1[r]:rp1[r + 1]], val1[rp1[r]:rp1[r + 1]])
        b = (col2[rp2[r]:rp2[r + 1]], val2[rp2[r]:rp2[r + 1]])
        if not (np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])):
            differ.add(r // rows_per_layer)
    # index change between layers 2 and 3: rows of layers 1..4 may change
    assert differ and differ <= {1, 2, 3, 4}, differ
    assert {2, 3} <= differ


def _source(prob, rhs=0):
    nx, ny, nz = prob.shape
    d = I.direction_index(0, 0, 1)
    return I.Source(np.array([prob.state(nx // 2 + rhs % 2, ny // 2, 0, d),
                              prob.state(nx // 2, ny // 2 - rhs % 2, 1, I.direction_index(1, 0, 1))], np.int64),
                    np.array([1.0, 0.5]), rhs % 3, np.exp(-0.5 * ((np.arange(7) - 3.0) / 1.5) ** 2))


@pytest.mark.parametrize("name,prob,steps,tol", [
    ("contrast_fp64", cases()[1][1], 120, 1e-12),
    ("thin_middle_mirror_fp32", cases()[3][1], 300, 1e-5),
    ("layers12_fp32", cases()[0][1], 300, 1e-5),
])
def test_two_step_steps_match_oracle(gpu, oracle_mod, name, prob, steps, tol):
    src = _source(prob)
    csr = oracle_mod.assemble(prob)
    ci = oracle_mod.column_info(prob)
    xo, deto, ledo = oracle_mod.run(prob, csr, steps, src.as_tuple(), colinfo=ci)
    with gpu.Context(prob, max_steps=steps) as ctx:
        ctx.set_source(0, src)
        ctx.step_n(steps)
        x = ctx.read_state()
        det, led = ctx.read_detectors()
    e = rel_l1(x, xo)
    print(f"two-step {name} rel L1 after {steps} steps: {e:.3e}")
    assert e <= tol, e
    assert rel_l1(det, deto) <= tol
    led_tol = 1e-11 if prob.precision == I.FP64 else 1e-4
    assert np.allclose(led, ledo, rtol=led_tol, atol=1e-13), (led, ledo)
    # mass balance: what is in the grid + absorbed + exited = injected
    assert led[0] + led[2] + led[3] == pytest.approx(led[1], rel=max(tol, 1e-11))


@pytest.mark.parametrize("kernel,n_rhs", [(0, 5), (1, 6), (1, 64)])
def test_two_step_batched_matches_oracle(gpu, oracle_mod, kernel, n_rhs):
    """Batched FP32 steps (CUDA-core and tensor-core forms) of the three-layer
    problem with two-step interfaces, each right-hand side against the oracle
    run alone."""
    prob, _ = I.three_layers(12, precision=I.FP32)
    prob.interface = I.INTERFACE_TWO_STEP
    prob.n_rhs = n_rhs
    prob.batched_kernel = kernel
    srcs = [_source(prob, r) for r in range(n_rhs)]
    steps = 60
    csr = oracle_mod.assemble(prob)
    ci = oracle_mod.column_info(prob)
    with gpu.Context(prob, max_steps=steps) as ctx:
        for r, s in enumerate(srcs):
            ctx.set_source(r, s)
        ctx.step_n(steps)
        picks = sorted({0, 1, n_rhs // 2, n_rhs - 1})
        got = {r: (ctx.read_state(r),) + tuple(ctx.read_detectors(r)) for r in picks}
    tol = 1e-5 if kernel == 0 else 1e-4
    for r, (x, det, led) in got.items():
        xo, deto, ledo = oracle_mod.run(prob, csr, steps, srcs[r].as_tuple(), colinfo=ci)
        assert rel_l1(x, xo) < tol, (r, rel_l1(x, xo))
        assert rel_l1(det, deto) < tol, r
        assert np.allclose(led, ledo, rtol=tol, atol=1e-12), (r, led, ledo)


def test_two_step_rejects_non_layered_media(gpu):
    prob = cases()[1][1]
    mov = np.array(prob.medium_of_voxel)
    mov[4, 2, 3] = 0
    bad = copy.copy(prob)
    bad.medium_of_voxel = mov
    with pytest.raises(gpu.DrtsError, match="one medium per z layer"):
        gpu.Context(bad)
    bad = copy.copy(prob)
    bad.interface = 2
    with pytest.raises(gpu.DrtsError, match="bad interface"):
        gpu.Context(bad)
