"""Precision tiers at the configurations' run lengths, against the FP64 oracle.

The configurations step 1000-5000 times; rounding that is biased (the
stored matrix is the same stencil in every interior voxel) adds up linearly
over a run, so each tier is checked at the length it is used for:
  * FP32 plain step, three layers at 48^3, 1000 steps: relative L1 <= 1e-5;
  * FP16-rowscale plain step, 24^3 inclusions, 1500 steps: <= 1e-4;
  * batched FP32 and batched FP16-rowscale, 24^3 inclusions x 8
    right-hand sides, 1500 steps: <= 1e-4 for every checked right-hand side;
  * the tensor-core batched step (block-floating bf16 terms, tcgen05), the
    same problem and length: <= 1e-4.
Each test prints the measured error.
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


def test_fp32_three_layers_48_1000_steps(gpu, oracle_mod):
    """FP32 tolerance of 1e-5 per 1000 steps on a grid of 2.9M states and
    0.59G nonzeros (every layer 4-36 voxels thick), Gaussian pulse."""
    prob, src = I.three_layers(48, precision=I.FP32)
    steps = 1000
    csr = oracle_mod.assemble(prob)
    xo, deto, ledo = oracle_mod.run(prob, csr, steps, src.as_tuple())
    del csr
    with gpu.Context(prob, max_steps=steps) as ctx:
        ctx.set_source(0, src)
        ctx.autotune(2)
        ctx.step_n(steps)
        x = ctx.read_state()
        det, led = ctx.read_detectors()
    e = rel_l1(x, xo)
    print(f"FP32 48^3 three layers rel L1 after {steps} steps: {e:.3e}")
    assert e <= 1e-5
    assert rel_l1(det, deto) <= 1e-5
    assert np.allclose(led, ledo, rtol=1e-5, atol=1e-12)


def test_fp16_plain_inclusions_1500_steps(gpu, oracle_mod):
    prob, srcs = I.inclusions(24, n_rhs=1, seed=3, precision=I.FP16_ROWSCALE)
    steps = 1500
    csr = oracle_mod.assemble(prob)
    xo, deto, ledo = oracle_mod.run(prob, csr, steps, srcs[0].as_tuple())
    with gpu.Context(prob, max_steps=steps) as ctx:
        ctx.set_source(0, srcs[0])
        ctx.step_n(steps)
        x = ctx.read_state()
        det, led = ctx.read_detectors()
    e = rel_l1(x, xo)
    print(f"FP16-rowscale plain 24^3 inclusions rel L1 after {steps} steps: {e:.3e}")
    assert x.min() >= 0.0
    assert e <= 1e-4
    assert rel_l1(det, deto) <= 1e-4
    assert np.allclose(led, ledo, rtol=1e-4, atol=1e-12)


@pytest.mark.parametrize("precision,kernel", [(I.FP32, 0), (I.FP16_ROWSCALE, 0), (I.FP32, 1)],
                         ids=["fp32", "fp16", "tensor"])
def test_batched_inclusions_1500_steps(gpu, oracle_mod, precision, kernel):
    prob, srcs = I.inclusions(24, n_rhs=8, seed=3, precision=precision)
    prob.batched_kernel = kernel
    steps = 1500
    csr = oracle_mod.assemble(prob)
    ci = oracle_mod.column_info(prob)
    with gpu.Context(prob, max_steps=steps) as ctx:
        for r, s in enumerate(srcs):
            ctx.set_source(r, s)
        ctx.step_n(steps)
        xs = [ctx.read_state(r) for r in range(8)]
        dets = [ctx.read_detectors(r) for r in range(8)]
    name = ("FP32" if precision == I.FP32 else "FP16-rowscale") + (" tensor-core" if kernel else "")
    for r in (0, 3, 5):
        xo, deto, ledo = oracle_mod.run(prob, csr, steps, srcs[r].as_tuple(), colinfo=ci)
        e = rel_l1(xs[r], xo)
        print(f"batched {name} 24^3 x 8 rhs {r} rel L1 after {steps} steps: {e:.3e}")
        assert e <= 1e-4, (r, e)
        assert rel_l1(dets[r][0], deto) <= 1e-4, r
        assert np.allclose(dets[r][1], ledo, rtol=1e-4, atol=1e-12), (r, dets[r][1], ledo)
