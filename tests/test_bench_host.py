"""Host-side arithmetic of bench.py on CPU: algorithmic bytes of a step, the
ncu traffic file tied to the step kernel's source, and the launch count the
batched line claims."""
import json
import types

import pytest

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
    """Each committed capture scales to a launch by nonzeros when it was
    taken on the current kernel source, for its own precision and variant;
    no capture, no traffic figure."""
    nnz = 11429626472
    caps = bench.traffic_captures()
    assert caps
    for d in caps:
        if d["kernel_sha"] != bench.kernel_hash():
            assert bench.traffic_per_launch("three_layers_128", d["precision"], nnz, d["variant"]) is None or any(
                c["kernel_sha"] == bench.kernel_hash() and c["precision"] == d["precision"]
                and c["variant"] == d["variant"] for c in caps)
            continue
        t = bench.traffic_per_launch("three_layers_128", d["precision"], nnz, d["variant"])
        assert t == d["dram_bytes_per_nnz"] * nnz
        # bytes per nonzero: the algorithmic ones plus slice padding (FP32:
        # 4 B value + 2 B code; FP16: 2 + 2 B and the second terms of split
        # values, per nonzero of the matrix)
        lo, hi = {"fp32": (6.0, 6.5), "fp16": (4.0, 4.5)}[d["precision"]]
        assert lo < d["dram_bytes_per_nnz"] < hi
    assert bench.traffic_per_launch("three_layers_128", "fp64", nnz) is None
    # a variant without a capture has no traffic figure
    assert bench.traffic_per_launch("three_layers_128", "fp32", nnz, 5) is None


def test_batched_launch_count():
    args = types.SimpleNamespace(batched_kernel="cuda", steps=5)
    info = _info(1, 1, n_patch=4)
    # detector + ledger + one product launch per tile of 8 (64 / 8)
    assert bench.batched_launches(args, {"variant": 0, "rhs_tile": 8}, info, 64) == (2 + 8) * 5
    # the halo order and the tensor-core form run the product in one launch
    assert bench.batched_launches(args, {"variant": 2, "rhs_tile": 4}, info, 64) == 3 * 5
    args.batched_kernel = "tensor"
    assert bench.batched_launches(args, {"variant": 0, "rhs_tile": 16}, info, 64) == 3 * 5
    # the tensor-core form needs no tuning record to count its launches
    assert bench.batched_launches(args, None, info, 64) == 3 * 5
    # the CUDA-core form without a tuning record has no known count
    args.batched_kernel = "cuda"
    assert bench.batched_launches(args, None, info, 64) is None
    # no detector patches: no detector launch
    assert bench.batched_launches(args, {"variant": 1, "rhs_tile": 4}, _info(1, 1, 0), 6) == (1 + 2) * 5


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference (the oracle timed on the host cores) prints
    exactly one JSON line with the keys of the benchmark contract."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                        "three_layers_16", "--steps", "2", "--warmup", "3"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 2 and d["warmup"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    # fewer than three warm-up steps are raised to three (the timing rule)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                        "three_layers_16", "--steps", "1", "--warmup", "1"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and json.loads(r.stdout.strip().splitlines()[-1])["warmup"] == 3


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the reference arm; the other ranks
    exit 0 without work or output."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                        "three_layers_16", "--steps", "1", "--warmup", "3", "--gpus", "2"],
                       cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_clock_summary_reads_nvidia_smi_rows():
    cs = bench.ClockSampler(0)
    assert cs.summary()["reasons"] == ["no samples"]
    idle = ["0", "2070", "2070", "310.2", "0x0000000000000000", "Not Active", "Not Active",
            "Not Active", "Not Active"]
    capped = ["0", "1965", "2070", "1398.7", "0x0000000000000004", "Not Active", "Not Active",
              "Not Active", "Active"]
    cs.samples = [idle, capped, capped, ["0", "[N/A]", "[N/A]", "[N/A]", "[N/A]"]]
    s = cs.summary()
    assert s["sm_mhz"] == 1965.0 and s["sm_max_mhz"] == 2070.0      # median of the readable ones
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4
    hot = list(capped)
    hot[7] = "Active"                                                # sw_thermal_slowdown
    cs.samples = [hot]
    assert cs.summary()["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]


def test_peaks_prefer_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6787.6}))
    assert bench.peaks() == (6787.6, "measured")


def test_batched_roofline_counts_the_methods_work():
    """The batched roofline counts 2 x nnz x R flops (one multiply-add per
    nonzero and right-hand side, no compensation terms) and A once plus every
    state read and written once; the binding roof is the slower of the FP32
    FMA roof and the HBM roof, and the FMA peak follows the device's SM count."""
    info = _info(4_799_000_000, 23_003_136)
    R = 64
    flops = 2.0 * info.nnz * R
    nbytes = bench.batched_bytes(info, "fp32", R)
    assert nbytes == info.nnz * 6 + 2 * info.n_states * R * 4
    peak = bench.fp32_fma_peak_tflops(152, 2070.0)
    assert peak == pytest.approx(80.55, rel=1e-3)
    assert bench.fp32_fma_peak_tflops(148, 2070.0) < peak
    r = bench.batched_roofline(flops, nbytes, 90.0, peak, 6787.6, "cuda")
    assert r["bound"] == "alu"
    assert r["frac"] == pytest.approx(flops / (peak * 1e12) / 0.090, rel=1e-3)
    assert r["achieved"] == pytest.approx(flops / 0.090 / 1e12, rel=1e-3)
    # a single right-hand side is HBM-bound
    r1 = bench.batched_roofline(2.0 * info.nnz, bench.batched_bytes(info, "fp32", 1), 5.0, peak,
                                6787.6, "cuda")
    assert r1["bound"] == "hbm" and r1["unit"] == "GB/s"


def test_config_workloads():
    """``--workload config:<name>`` builds the JSON problem file's workload,
    the same problem as the generator name it stands for."""
    import numpy as np
    p, s = bench.workload("config:plain_fp64_cube16", "fp64")
    q, t = bench.workload("fresnel_cube_16", "fp64")
    assert p.shape == q.shape and p.media == q.media and np.array_equal(s.state, t.state)
    pb, srcs = bench.workload("config:batched_inclusions96x64", "fp32")
    assert pb.n_rhs == 64 and len(srcs) == 64
