"""drts_state_sum_noalloc: the state-mass sum for callers that cannot
allocate device memory when they need it (real-time loops that must not wait
on the allocator, processes whose device memory is owned by another
runtime's pool).  It must agree with the sum returned by drts_read_detectors,
which allocates its own result buffer, on two calls in a row, for one
right-hand side and for the batched layout that keeps right-hand sides in
groups of four.  The file name makes pytest collect it last."""
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
    torch.cuda.set_device(0)
    return torch, drts


def test_state_sum_noalloc_matches_ledger_sum(gpu):
    torch, drts = gpu
    stream = torch.cuda.current_stream()
    prob, src = I.three_layers(20, precision=I.FP32)
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")   # caller-owned output
    with drts.Context(prob, max_steps=40, stream=stream.cuda_stream) as ctx:
        ctx.set_source(0, src)
        for call in range(2):
            ctx.step_n(20)
            _, led = ctx.read_detectors()            # reference: allocating path
            ctx.state_sum_noalloc(out.data_ptr() + 8 * call)
            torch.cuda.synchronize()
            got = float(out[call].item())
            assert led[0] > 0.0
            assert got == pytest.approx(led[0], rel=1e-12), (call, got, led[0])
        # the sum of the host copy of the state agrees too
        x = ctx.read_state()
        assert float(out[1].item()) == pytest.approx(float(np.sum(x)), rel=1e-12)


def test_state_sum_noalloc_batched_grouped_layout(gpu):
    """Six right-hand sides: two groups of four, the second ragged; the sum
    of every right-hand side (offset r % 4 in its group, stride 4) equals the
    ledger's, on two calls in a row."""
    torch, drts = gpu
    stream = torch.cuda.current_stream()
    R = 6
    prob, srcs = I.inclusions(12, n_rhs=R, precision=I.FP32)
    out = torch.full((2, R), -1.0, dtype=torch.float64, device="cuda")
    with drts.Context(prob, max_steps=30, stream=stream.cuda_stream) as ctx:
        for r, s in enumerate(srcs):
            ctx.set_source(r, s)
        for call in range(2):
            ctx.step_n(15)
            ref = [ctx.read_detectors(r)[1][0] for r in range(R)]
            for r in range(R):
                ctx.state_sum_noalloc(out.data_ptr() + 8 * (call * R + r), rhs=r)
            torch.cuda.synchronize()
            got = out[call].cpu().numpy()
            for r in range(R):
                assert ref[r] > 0.0
                assert got[r] == pytest.approx(ref[r], rel=1e-12), (call, r, got[r], ref[r])
        for r in (0, 5):
            assert float(out[1, r].item()) == pytest.approx(float(np.sum(ctx.read_state(r))), rel=1e-12)
