"""Host-side arithmetic of bench.py on CPU: algorithmic bytes of a step, the
ncu traffic file tied to the step kernel's source, and the launch count the
batched line claims."""
import json
import types

import bench


def _info(nnz, n_states, n_patch=256, nnz_stored=None):
    return types.SimpleNamespace(nnz=nnz, n_states=n_states, n_patch=n_patch,
                                 nnz_stored=nnz if nnz_stored is None else nnz_stored)


def test_algorithmic_bytes_per_precision():
    info = _info(1000, 100)
    # values + 16-bit codes per nonzero, x read and y written once per state
    assert bench.algorithmic_bytes(info, "fp32") == 1000 * 6 + 2 * 100 * 4
    assert bench.algorithmic_bytes(info, "fp64") == 1000 * 10 + 2 * 100 * 8
    # FP16 values, FP32 state, plus a 4-byte row scale per row; the stored
    # entries include the second terms of split values
    info16 = _info(1000, 100, nnz_stored=1020)
    assert bench.algorithmic_bytes(info16, "fp16") == 1020 * 4 + 2 * 100 * 4 + 100 * 4


def test_traffic_follows_kernel_source():
    d = json.load(open(bench.TRAFFIC_FILE))
    nnz = 11429626472
    if d["kernel_sha"] == bench.kernel_hash():
        t = bench.traffic_per_launch("three_layers_128", d["precision"], nnz)
        assert t == d["dram_bytes_per_nnz"] * nnz
        # the capture's bytes per nonzero are the algorithmic ones plus padding
        assert 6.0 < d["dram_bytes_per_nnz"] < 6.5
    assert bench.traffic_per_launch("three_layers_128", "fp64", nnz) is None


def test_batched_launch_count():
    args = types.SimpleNamespace(batched_kernel="cuda", steps=5)
    info = _info(1, 1, n_patch=4)
    # detector + ledger + one product launch per tile of 8 (64 / 8)
    assert bench.batched_launches(args, {"variant": 0, "rhs_tile": 8}, info, 64) == (2 + 8) * 5
    # the halo order and the tensor-core form run the product in one launch
    assert bench.batched_launches(args, {"variant": 2, "rhs_tile": 4}, info, 64) == 3 * 5
    args.batched_kernel = "tensor"
    assert bench.batched_launches(args, {"variant": 0, "rhs_tile": 16}, info, 64) == 3 * 5
    assert bench.batched_launches(args, None, info, 64) is None
    # no detector patches: no detector launch
    args.batched_kernel = "cuda"
    assert bench.batched_launches(args, {"variant": 1, "rhs_tile": 4}, _info(1, 1, 0), 6) == (1 + 2) * 5
