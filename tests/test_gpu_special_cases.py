"""Degenerate and extreme cases of the CUDA path, through the C ABI, checked
against closed forms the method fixes (no oracle needed) or the oracle:
ballistic translation with no scattering (value 1.0 exactly), exponential
decay in a closed box, and the largest batch (64 right-hand sides)."""
import math

import numpy as np
import pytest

from paper_1611_08536_gb300 import inputs as I

pytestmark = pytest.mark.gpu

D = I.direction_index


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_08536_gb300 import build, drts
    build.build()
    drts.load()
    return drts


@pytest.mark.parametrize("precision", [I.FP64, I.FP32, I.FP16_ROWSCALE])
def test_ballistic_translation_exact(gpu, precision):
    """mu_s = mu_a = 0, one medium: the axis stencil has a single target of
    weight exactly 1 (Eq. 18 with L = h), so a delta pulse moves one voxel per
    step along +z with value 1.0 and nothing anywhere else."""
    n = 12
    prob = I.Problem((6, 6, n), 0.1, [(0.0, 0.0, 0.0, 1.3)], np.zeros((n, 6, 6), np.uint8), 1.0,
                     I.MIRROR, precision, 1, I.FACE_PZ, 2, 2, "ballistic")
    d = D(0, 0, 1)
    src = I.Source(np.array([prob.state(3, 2, 0, d)], np.int64), np.ones(1), 0, np.ones(1))
    with gpu.Context(prob, max_steps=n) as ctx:
        ctx.set_source(0, src)
        for k in range(1, n):
            ctx.step_n(1)
            x = ctx.read_state()
            expect = np.zeros(prob.n_states)
            expect[prob.state(3, 2, k - 1, d)] = 1.0
            assert np.array_equal(x, expect), k


@pytest.mark.parametrize("precision,tol", [(I.FP64, 1e-13), (I.FP32, 5e-6)])
def test_pure_decay_closed_box(gpu, precision, tol):
    """mu_s = 0, mirror box: the total population decays as exp(-mu_a L t)
    exactly (Eq. 8); the ledger's absorbed mass closes the balance."""
    mu_a, h = 0.7, 0.1
    prob = I.Problem((5, 4, 6), h, [(0.0, mu_a, 0.0, 1.4)], np.zeros((6, 4, 5), np.uint8), 1.0,
                     I.MIRROR, precision, 1, I.FACE_PZ, 2, 2, "decay")
    src = I.Source(np.array([prob.state(2, 1, 3, D(1, -1, 1)), prob.state(0, 0, 0, D(0, 1, 0))],
                            np.int64), np.array([0.25, 0.75]), 0, np.ones(1))
    T = 40
    with gpu.Context(prob, max_steps=T) as ctx:
        ctx.set_source(0, src)
        ctx.step_n(T)
        x = ctx.read_state()
        _, led = ctx.read_detectors()
    expect = math.exp(-mu_a * h * (T - 1))       # injected at t = 0, lands in x(1)
    assert x.sum() == pytest.approx(expect, rel=tol)
    assert led[0] + led[2] + led[3] == pytest.approx(led[1], rel=tol)
    assert led[3] == 0.0


def test_batched_64_rhs(gpu, oracle_mod):
    """The largest batch: 64 right-hand sides in one context (16 passes of 4,
    or 8 of 8) against the oracle run alone for a spread of them."""
    prob, srcs = I.inclusions(12, n_rhs=64, seed=33, precision=I.FP32, n_spheres=2)
    steps = 25
    csr = oracle_mod.assemble(prob)
    with gpu.Context(prob, max_steps=steps) as ctx:
        for r, s in enumerate(srcs):
            ctx.set_source(r, s)
        ctx.step_n(steps)
        xs = {r: ctx.read_state(r) for r in (0, 17, 38, 63)}
    for r, x in xs.items():
        xo, _, _ = oracle_mod.run(prob, csr, steps, srcs[r].as_tuple())
        assert np.abs(x - xo).sum() / np.abs(xo).sum() < 1e-5, r


@pytest.mark.parametrize("precision", [I.FP32, I.FP16_ROWSCALE])
def test_assembly_survives_every_failed_allocation(gpu, oracle_mod, precision):
    """Host-side allocator fault: the k-th device allocation of a context
    fails, for every k the assembly reaches.  Each failure returns
    DRTS_ENOMEM with nothing left allocated (repeated failures do not grow the
    device memory in use), and the first k past the last allocation
    assembles a context whose step matches the oracle."""
    import torch
    prob, _ = I.three_layers(8, precision=precision)
    free = []
    try:
        for k in range(200):
            gpu.set_alloc_fault(k)
            try:
                ctx = gpu.Context(prob, max_steps=4)
            except gpu.DrtsError as e:
                assert e.status == gpu.ENOMEM, (k, e)
                torch.cuda.synchronize()
                free.append(torch.cuda.mem_get_info()[0])
                continue
            break
        else:
            pytest.fail("the assembly never completed")
    finally:
        gpu.set_alloc_fault(-1)
    assert len(free) >= 5
    # device memory free after the last failure vs after the fourth
    assert free[-1] >= free[3] - (8 << 20), (free[3], free[-1])
    with ctx:
        rng = np.random.default_rng(2)
        x0 = rng.random(prob.n_states)
        ctx.write_state(x0)
        ctx.step_n(1)
        x1 = ctx.read_state()
    y = oracle_mod.spmv(oracle_mod.assemble(prob), x0)
    tol = 1e-6 if precision == I.FP32 else 2e-3
    assert np.abs(x1 - y).sum() / np.abs(y).sum() < tol


def test_torch_caching_allocator_owns_context_buffers(gpu, oracle_mod):
    """With drts_set_allocator pointed at PyTorch's caching allocator the
    context's device buffers are PyTorch's (counted by
    torch.cuda.memory_allocated, returned on close) and the step is the same."""
    import torch
    prob, _ = I.three_layers(10, precision=I.FP32)
    rng = np.random.default_rng(8)
    x0 = rng.random(prob.n_states)
    before = torch.cuda.memory_allocated()
    try:
        gpu.use_torch_allocator()
        with gpu.Context(prob, max_steps=2) as ctx:
            held = torch.cuda.memory_allocated() - before
            assert held >= ctx.info().matrix_bytes
            ctx.write_state(x0)
            ctx.step_n(1)
            x1 = ctx.read_state()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
    finally:
        gpu.use_cuda_allocator()
    y = oracle_mod.spmv(oracle_mod.assemble(prob), x0)
    assert np.abs(x1 - y).sum() / np.abs(y).sum() < 1e-6
