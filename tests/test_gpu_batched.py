"""Batched step X(t+1) = A X(t) + S(t): every right-hand side must match the
FP64 oracle run alone, and the single-RHS path of the same problem."""
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


def run_batched(gpu, prob, srcs, steps, tile=0, order=-1):
    with gpu.Context(prob, max_steps=steps) as ctx:
        if tile or order >= 0:
            ctx.set_launch(0, 0, tile, order)
        for r, s in enumerate(srcs):
            ctx.set_source(r, s)
        ctx.step_n(steps)
        xs, dets, leds = [], [], []
        for r in range(len(srcs)):
            xs.append(ctx.read_state(r))
            d, l = ctx.read_detectors(r)
            dets.append(d)
            leds.append(l)
    return xs, dets, leds


@pytest.mark.parametrize("n_rhs,tile,order", [(5, 0, -1), (5, 4, 0), (8, 8, 0), (13, 16, 0), (33, 32, 0),
                                              (5, 4, 1), (8, 8, 1), (13, 16, 1), (33, 32, 1),
                                              (2, 4, 2), (5, 4, 2), (13, 4, 2), (33, 4, 2)])
def test_batched_fp32_matches_oracle(gpu, oracle_mod, n_rhs, tile, order):
    """All slice orders (warps striding over slices; block-major; block-major
    with the x halo in shared memory) and every right-hand-side tile, on a
    12^3 grid whose 54 voxel blocks of 32 wrap across x rows (ragged block
    boundaries, halo ranges reaching past both ends of the state)."""
    prob, srcs = I.inclusions(12, n_rhs=n_rhs, seed=21, precision=I.FP32, n_spheres=2)
    steps = 40
    csr = oracle_mod.assemble(prob)
    ci = oracle_mod.column_info(prob)
    xs, dets, leds = run_batched(gpu, prob, srcs, steps, tile, order)
    for r in range(0, n_rhs, max(1, n_rhs // 5)):
        xo, deto, ledo = oracle_mod.run(prob, csr, steps, srcs[r].as_tuple(), colinfo=ci)
        assert rel_l1(xs[r], xo) < 1e-5, r
        assert rel_l1(dets[r], deto) < 1e-5, r
        assert np.allclose(leds[r], ledo, rtol=1e-5, atol=1e-12), (r, leds[r], ledo)


def test_batched_same_alone_and_in_mix(gpu):
    prob, srcs = I.inclusions(14, n_rhs=6, seed=5, precision=I.FP32, n_spheres=2)
    steps = 30
    xs, dets, _ = run_batched(gpu, prob, srcs, steps)
    import copy
    for r in (0, 3, 5):
        p1 = copy.copy(prob)
        p1.n_rhs = 1
        x1, d1, _ = run_batched(gpu, p1, [srcs[r]], steps)
        assert rel_l1(xs[r], x1[0]) < 1e-6
        assert rel_l1(dets[r], d1[0]) < 1e-6


@pytest.mark.parametrize("order", [0, 1, 2])
def test_batched_fp64_and_fp16(gpu, oracle_mod, order):
    for prec, tol in ((I.FP64, 1e-12), (I.FP16_ROWSCALE, 1e-4)):
        prob, srcs = I.inclusions(10, n_rhs=4, seed=8, precision=prec, n_spheres=1)
        steps = 20
        csr = oracle_mod.assemble(prob)
        xs, _, _ = run_batched(gpu, prob, srcs, steps, 4, order)
        for r in range(4):
            xo, _, _ = oracle_mod.run(prob, csr, steps, srcs[r].as_tuple())
            assert rel_l1(xs[r], xo) < tol, (prec, r)


def test_batched_fp16_500_steps(gpu, oracle_mod):
    """Batched FP16-rowscale step (FP32 state and accumulation) on a 24^3
    cube with absorbing inclusions, 8 right-hand sides, 500 steps: every
    checked right-hand side within 1e-4 of the FP64 oracle."""
    prob, srcs = I.inclusions(24, n_rhs=8, seed=3, precision=I.FP16_ROWSCALE)
    steps = 500
    csr = oracle_mod.assemble(prob)
    ci = oracle_mod.column_info(prob)
    xs, dets, _ = run_batched(gpu, prob, srcs, steps)
    for r in (0, 5):
        xo, deto, _ = oracle_mod.run(prob, csr, steps, srcs[r].as_tuple(), colinfo=ci)
        e = rel_l1(xs[r], xo)
        print(f"batched FP16 rhs {r} rel L1 after {steps} steps: {e:.3e}")
        assert e < 1e-4, (r, e)
        assert rel_l1(dets[r], deto) < 1e-4, r


@pytest.mark.parametrize("n_rhs", [3, 8, 20, 64])
def test_tensor_core_batched_matches_oracle(gpu, oracle_mod, n_rhs):
    """Tensor-core batched step (bf16 high/low splits, FP32 accumulation):
    every right-hand side against the FP64 oracle."""
    prob, srcs = I.inclusions(12, n_rhs=n_rhs, seed=21, precision=I.FP32, n_spheres=2)
    prob.batched_kernel = gpu.BATCHED_TENSOR
    steps = 40
    csr = oracle_mod.assemble(prob)
    ci = oracle_mod.column_info(prob)
    xs, dets, leds = run_batched(gpu, prob, srcs, steps)
    worst = 0.0
    for r in range(0, n_rhs, max(1, n_rhs // 4)):
        xo, deto, ledo = oracle_mod.run(prob, csr, steps, srcs[r].as_tuple(), colinfo=ci)
        e = rel_l1(xs[r], xo)
        worst = max(worst, e)
        assert e < 1e-4, (r, e)
        assert rel_l1(dets[r], deto) < 1e-4, r
        assert np.allclose(leds[r], ledo, rtol=1e-4, atol=1e-12), (r, leds[r], ledo)
    print(f"tensor-core batched rel L1 after {steps} steps (worst rhs): {worst:.3e}")


def test_tensor_core_batched_same_alone_and_in_mix(gpu):
    prob, srcs = I.inclusions(12, n_rhs=6, seed=5, precision=I.FP32, n_spheres=2)
    prob.batched_kernel = gpu.BATCHED_TENSOR
    xs, dets, _ = run_batched(gpu, prob, srcs, 25)
    import copy
    p1 = copy.copy(prob)
    p1.n_rhs = 2
    for r in (0, 4):
        x1, d1, _ = run_batched(gpu, p1, [srcs[r], srcs[(r + 1) % 6]], 25)
        assert rel_l1(xs[r], x1[0]) < 1e-6
        assert rel_l1(dets[r], d1[0]) < 1e-6


def test_tensor_core_ragged_grid_and_rejections(gpu, oracle_mod):
    """Tensor-core batched step on a ragged 5 x 7 x 3 grid with mirror and
    Fresnel edges mixed through two media (every line of the sweep has
    missing neighbour lines), 3 right-hand sides; sub-step sources are
    rejected for this form."""
    mov = np.zeros((3, 7, 5), np.uint8)
    mov[:, 4:, :] = 1
    prob = I.Problem((5, 7, 3), 0.1, [(8.0, 0.05, 0.85, 1.4), (12.0, 0.02, 0.9, 1.4)], mov, 1.0,
                     I.FRESNEL, I.FP32, 3, I.FACE_PZ, 2, 3, "ragged_tc")
    prob.batched_kernel = gpu.BATCHED_TENSOR
    srcs = [I.Source(np.array([prob.state(1 + r, 2 + r, 0, I.direction_index(0, 0, 1))], np.int64),
                     np.ones(1), 0, np.ones(1)) for r in range(3)]
    steps = 60
    csr = oracle_mod.assemble(prob)
    xs, dets, leds = run_batched(gpu, prob, srcs, steps)
    for r in range(3):
        xo, deto, ledo = oracle_mod.run(prob, csr, steps, srcs[r].as_tuple())
        assert rel_l1(xs[r], xo) < 1e-4, r
        assert rel_l1(dets[r], deto) < 1e-4, r
        assert np.allclose(leds[r], ledo, rtol=1e-4, atol=1e-12), (r, leds[r], ledo)
    with gpu.Context(prob, max_steps=4) as ctx:
        with pytest.raises(gpu.DrtsError) as e:
            ctx.inject_source_substeps(0, [0], [1.0], 0, np.ones((1, 2)))
        assert e.value.status == gpu.EUNSUPPORTED
