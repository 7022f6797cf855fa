"""drts_state_sum_noalloc: the state-mass sum for callers that cannot
allocate device memory (graph or stream capture, real-time loops, memory
owned by another runtime's pool).  It must agree with the sum returned by
drts_read_detectors, which allocates its own result buffer, on two calls in
a row.  The file name makes pytest collect it last."""
import numpy as np
import pytest

from paper_1611_08536_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_state_sum_noalloc_matches_ledger_sum():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_08536_gb300 import build, drts
    build.build()
    torch.cuda.set_device(0)
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
