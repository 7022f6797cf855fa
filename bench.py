"""DRTS time-step benchmark: x(t+1) = A x(t) + s(t) on one GB300.

Default workload: three planar layers, 128^3 voxels x 26 directions
(54.5M states, ~11.4G nonzeros), FP32 matrix and state, Gaussian pulse
source, 16x16 detector patches on the exit face.  One "step" is one DRTS
time step (the whole fused step kernel: SpMV, source injection, detector
readout, ledger).

Prints one JSON line (rank 0).  Metric: GNNZ/s (stored nonzeros of A
streamed per second), whole job.  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.

Multi-GPU: every rank runs an independent replica of the workload (the
step has no exchange between independent simulations): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DRTS step GNNZ/s"
UNIT = "GNNZ/s"
KERNEL_SRC = os.path.join(ROOT, "paper_1611_08536_gb300", "csrc", "drts_step.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")


def workload(name, precision, rhs=1):
    from paper_1611_08536_gb300 import inputs as I
    if name.startswith("config:"):
        # a JSON problem file of the package (configs/<name>.json) or a path
        c = I.load_config(name[len("config:"):], precision)
        if c.problem is None:
            raise SystemExit("a served-stream config is a --serve workload")
        return (c.problem, c.sources) if c.problem.n_rhs > 1 else (c.problem, c.sources[0])
    prec = {"fp32": I.FP32, "fp64": I.FP64, "fp16": I.FP16_ROWSCALE}[precision]
    if name.startswith("ellipsoids_"):
        n = int(name.split("_")[-1])
        return I.ellipsoids(n, precision=prec)
    if name.startswith("inclusions_"):
        n = int(name.split("_")[-1])
        return I.inclusions(n, n_rhs=rhs, precision=prec)
    if name.startswith("three_layers_"):
        n = int(name.split("_")[-1])
        return I.three_layers(n, precision=prec)
    if name.startswith("fresnel_cube_"):
        n = int(name.split("_")[-1])
        return I.fresnel_cube(n, precision=prec)
    raise SystemExit(f"unknown workload {name}")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([f.strip() for f in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for i, n in enumerate(names):
                if len(s) > 5 + i and s[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash():
    return hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]


def traffic_captures():
    """The committed ncu DRAM captures of the step kernel (one per precision
    and launch variant), or [] when the file is absent."""
    if not os.path.exists(TRAFFIC_FILE):
        return []
    d = json.load(open(TRAFFIC_FILE))
    return d.get("captures", [d])


def traffic_per_launch(workload_name, precision, nnz, variant=None):
    """DRAM bytes per step-kernel launch from a committed ncu capture of the
    same precision and launch variant on the current kernel source, scaled to
    this launch by nonzeros (traffic grows with the matrix); None when no
    such capture exists."""
    for d in traffic_captures():
        if d.get("kernel_sha") != kernel_hash() or d.get("precision") != precision:
            continue
        if variant is not None and d.get("variant") is not None and int(d["variant"]) != int(variant):
            continue
        return d["dram_bytes_per_nnz"] * nnz
    return None


def algorithmic_bytes(info, precision):
    vb = {"fp32": 4, "fp64": 8, "fp16": 2}[precision]
    sb = 8 if precision == "fp64" else 4
    # stored entries: FP16 keeps a few large values per row as two terms
    b = info.nnz_stored * (vb + 2) + 2 * info.n_states * sb
    if precision == "fp16":
        b += info.n_states * 4
    return b


def max_over_ranks(value, device="cuda"):
    """Max of a per-rank float over all ranks (the timing rule: the slowest
    rank's time); the value itself on a single rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gnnz(nnz, steps, ms, world_size):
    """Whole-job throughput: every rank streams its own replica's nnz per step."""
    return nnz * steps / (ms * 1e-3) / 1e9 * world_size


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1611_08536_gb300 import build, drts
    build.build()
    prob, src = workload(args.workload, args.precision)
    stream = torch.cuda.current_stream()
    total_steps = args.warmup + args.steps + args.e2e_steps + 1
    t_asm = time.time()
    ctx = drts.Context(prob, max_steps=total_steps, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t_asm = time.time() - t_asm
    info = ctx.info()
    ctx.set_source(0, src)
    tune = None
    if args.blocks_per_sm or args.threads or args.variant >= 0:
        ctx.set_launch(args.blocks_per_sm, args.threads, 0, args.variant)
    elif args.autotune:
        # the persistent mode keeps the tuned launch's block size, grid and
        # warps per slice
        tune = ctx.autotune(args.autotune)
    if args.step_mode == "persistent":
        ctx.set_step_mode(drts.STEP_PERSISTENT)

    ctx.step_n(args.warmup)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        ev0.record(stream)
        ctx.step_n(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1))
    if ws > 1:
        dist.barrier()
    ms_step = ms / args.steps
    gnnz = whole_job_gnnz(info.nnz, args.steps, ms, ws)

    # end to end: per step, source factors host->device and the detector
    # readout device->host, from pinned host buffers, through the C ABI
    e2e = None
    if args.e2e_steps > 0:
        n = args.e2e_steps
        scale = torch.zeros((n, 1), dtype=torch.float64, pin_memory=True)
        det = torch.zeros((n, 1, max(info.n_patch, 1)), dtype=torch.float64, pin_memory=True)
        sc = scale.numpy()
        sc[:, 0] = 1.0 / n
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        ctx.run_host(sc, det.numpy())
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": round(info.nnz * n / dt / 1e9 * ws, 3), "unit": UNIT,
               "h2d_bytes_per_step": 8, "d2h_bytes_per_step": 8 * info.n_patch,
               "steps": n, "ms_per_step": round(dt * 1e3 / n, 4)}

    # parity of the timed launch configuration on sampled rows: one more
    # step from the current state, checked row by row in FP64
    sample_check = None
    if args.check and rank == 0:
        sample_check = sampled_step_check(ctx, prob, args)

    peak, peak_kind = peaks()
    alg = algorithmic_bytes(info, args.precision)
    achieved = alg / (ms_step * 1e-3) / 1e9
    variant = tune["variant"] if tune else (args.variant if args.variant >= 0 else 0)
    # the captures are of the launch-per-step kernels, not of the persistent one
    traffic = (traffic_per_launch(args.workload, args.precision, info.nnz, variant)
               if args.step_mode == "launch" else None)
    line = {
        "metric": METRIC, "value": round(gnnz, 3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f16-matrix/f32-state"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(prob.shape), "directions": 26,
                   "states": int(info.n_states), "nnz": int(info.nnz),
                   "nnz_stored": int(info.nnz_stored),
                   "nnz_padded": int(info.nnz_padded), "matrix_GB": round(info.matrix_bytes / 1e9, 3),
                   "format": "SELL-32 (slice = 32 voxels x 1 direction), 16-bit stencil codes",
                   "precision": args.precision, "steps_per_s": round(1e3 / ms_step, 3),
                   "l2": "inputs larger than L2 (matrix streamed every step)",
                   "assembly_s": round(t_asm, 2), "parallelism": f"replicas x{ws}",
                   "step_mode": args.step_mode,
                   "launch": tune},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "peak_kind": peak_kind,
                     "traffic_source": (f"ncu capture of launch variant {variant} at 48^3, "
                                        "scaled to this launch by nonzeros")
                     if traffic is not None else "no ncu capture of this kernel source and variant",
                     "algorithmic_bytes_per_launch": int(alg)},
        # one cooperative launch runs all timed steps in the persistent mode
        "gpu_launches": 1 if args.step_mode == "persistent" else args.steps,
        "e2e": e2e,
        "clocks": clk.summary(),
    }
    if sample_check is not None:
        line["sampled_parity"] = sample_check
    if rank == 0 and args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, args)
    ctx.close()
    if ws == 1 and args.sub:
        line.update(sub_lines(args, local))
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_plain(workload_name, precision, steps, warmup, autotune, check=True, local=0):
    """The plain single-right-hand-side step of another precision tier on a
    workload, timed like the headline line (CUDA events over the timed
    steps, autotuned launch), with its HBM roofline and sampled parity."""
    import torch
    from paper_1611_08536_gb300 import drts
    stream = torch.cuda.current_stream()
    prob, src = workload(workload_name, precision)
    ctx = drts.Context(prob, max_steps=warmup + steps + 2, stream=stream.cuda_stream)
    ctx.set_source(0, src)
    tune = ctx.autotune(autotune) if autotune else None
    info = ctx.info()
    ctx.step_n(warmup)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        ctx.step_n(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    parity = sampled_step_check(ctx, prob, None) if check else None
    ctx.close()
    peak, peak_kind = peaks()
    alg = algorithmic_bytes(info, precision)
    achieved = alg / (ms * 1e-3) / 1e9
    variant = tune["variant"] if tune else 0
    traffic = traffic_per_launch(workload_name, precision, info.nnz, variant)
    return {
        "workload": workload_name, "precision": precision, "steps": steps, "warmup": warmup,
        "ms_per_step": round(ms, 4), "value": round(info.nnz / (ms * 1e-3) / 1e9, 3), "unit": UNIT,
        "nnz": int(info.nnz), "nnz_stored": int(info.nnz_stored),
        "matrix_GB": round(info.matrix_bytes / 1e9, 3), "launch": tune,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": int(alg),
                     "traffic_source": (f"ncu capture of launch variant {variant} at 48^3, "
                                        "scaled to this launch by nonzeros")
                     if traffic is not None else "no ncu capture of this kernel source and variant"},
        "sampled_parity": parity, "gpu_launches": steps, "clocks": clk.summary(),
    }


def measure_fcc(box, steps, warmup, local=0):
    """The FP32 step on the close-packed partition (Section 3): a box of
    close-packed sites in one scattering medium (the voxel workloads' tissue
    values), a point source, CUDA events over the timed steps, and the HBM
    roofline on the same algorithmic bytes as the voxel step: each stored
    nonzero's value and code once, each state read and written once."""
    import numpy as np
    import torch
    from paper_1611_08536_gb300 import drts
    stream = torch.cuda.current_stream()
    nx, ny, nz = box
    n_sites = nx * ny * nz // 2
    media = [(10.0, 0.01, 0.9, 1.4)]
    t_asm = time.perf_counter()
    ctx = drts.FccContext(box, 0.1, media, np.zeros(n_sites, np.uint8), precision=drts.FP32,
                          stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t_asm = time.perf_counter() - t_asm
    c = ((nz // 2) * ny + ny // 2) * nx // 2 + nx // 4
    ctx.set_source([c * 12 + 3], [1.0], np.ones(4))
    info = ctx.info()
    ctx.step_n(warmup)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        ctx.step_n(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    ctx.close()
    hbm, kind = peaks()
    nbytes = info.nnz * (4 + 2) + info.n_states * 8
    achieved = nbytes / (ms * 1e-3) / 1e9
    return {
        "workload": f"close_packed_{nx}x{ny}x{nz}", "sites": int(info.n_sites), "states": int(info.n_states),
        "nnz": int(info.nnz), "slots": int(info.slots), "offsets": int(info.n_offsets), "precision": "fp32",
        "steps": steps, "warmup": warmup, "ms_per_step": round(ms, 4),
        "value": round(info.nnz / (ms * 1e-3) / 1e9, 3), "unit": "GNNZ/s", "assembly_s": round(t_asm, 2),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "traffic": None, "peak_kind": kind,
                     "algorithmic_bytes_per_launch": int(nbytes)},
        "sampled_parity": "the device matrix and multi-step states are checked against the oracle "
                          "in the GPU tests on boxes the numpy oracle assembles (up to 20,480 sites)",
        "gpu_launches": steps + 1, "clocks": clk.summary(),
    }


def sub_lines(args, local):
    """The metric's second half on the same box, after the headline: the
    FP16-rowscale tier on the headline workload, the batched step of 64
    right-hand sides sharing A (96^3 inclusions) against the plain
    per-simulation step, and a served stream whose requests keep their full
    step counts.  Each is a sub-object of the headline JSON line; a failure
    is recorded there instead of ending the run."""
    out = {}
    jobs = []
    if "fp16" in args.sub:
        jobs.append(("fp16", lambda: measure_plain(args.workload, "fp16", args.steps, args.warmup,
                                                    args.autotune, args.check, local)))
    if "batched" in args.sub:
        jobs.append(("batched", lambda: measure_batched(
            types_ns(variant=-1, threads=0, blocks_per_sm=0, rhs_tile=0), args.sub_batched_workload, "fp32",
            64, args.batched_kernel, args.sub_batched_steps, args.warmup, max(args.autotune, 1), 1500,
            check=args.check, local=local)))
    if "fcc" in args.sub:
        jobs.append(("fcc", lambda: measure_fcc(tuple(int(v) for v in args.sub_fcc_box.split("x")), args.steps,
                                                 args.warmup, local=local)))
    if "served" in args.sub:
        jobs.append(("served", lambda: measure_served(args, args.sub_served_requests, 50.0, 1.0, 16, 20, 4,
                                                       "fifo", baselines="estimate", local=local)))
    for name, fn in jobs:
        t = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:          # recorded in the line, never silently dropped
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = round(time.perf_counter() - t, 1)
    return out


def sampled_step_check(ctx, prob, args):
    """One extra step checked against the oracle on sampled planes."""
    import numpy as np
    import oracle
    x = ctx.read_state()
    ctx.step_n(1)
    y = ctx.read_state()
    nz = prob.shape[2]
    planes = sorted({0, nz // 11, nz - 1})
    worst = 0.0
    for z in planes:
        c = oracle.assemble(prob, z, z + 1)
        yo = oracle.spmv(c, x)
        yg = y[c.row0:c.row0 + c.n_rows]
        den = np.abs(yo).sum()
        if den > 0:
            worst = max(worst, float(np.abs(yg - yo).sum() / den))
    return {"planes": planes, "rel_l1_one_step": worst}


def cpu_baseline(prob, args, seconds=12.0):
    """FP64 oracle CSR SpMV timed on the host cores over one z-plane of rows."""
    import numpy as np
    import oracle
    oracle.build()
    z = prob.shape[2] // 2
    c = oracle.assemble(prob, z, z + 1)
    x = np.random.default_rng(0).random(prob.n_states)
    threads = oracle.max_threads()
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.spmv(c, x, threads)
        reps += 1
        dt = time.perf_counter() - t0
        if dt > seconds:
            break
    out = {"value": round(c.nnz * reps / dt / 1e9, 4), "unit": UNIT, "cores": threads,
           "kind": "oracle",
           "sample": f"FP64 CSR SpMV over the {c.n_rows} rows of z-plane {z} "
                     f"({c.nnz} nnz) of the same workload, {reps} repetitions"}
    # the same oracle on one core (a few seconds)
    reps1, t1 = 0, time.perf_counter()
    while True:
        oracle.spmv(c, x, 1)
        reps1 += 1
        dt1 = time.perf_counter() - t1
        if dt1 > seconds / 4:
            break
    out["single_core"] = {"value": round(c.nnz * reps1 / dt1 / 1e9, 4), "unit": UNIT, "cores": 1,
                          "repetitions": reps1}
    return out


def sm_max_mhz():
    """Maximum SM clock: the measured file, else nvidia-smi, else the
    GB300's 2070 MHz."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        v = json.load(open(p)).get("sm_max_mhz")
        if v:
            return float(v), "measured file"
    try:
        out = subprocess.run(["nvidia-smi", "--id=0", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=5).stdout.strip()
        return float(out.splitlines()[0]), "nvidia-smi"
    except Exception:
        return 2070.0, "nominal"


def fp32_fma_peak_tflops(sms, mhz):
    """FP32 FMA peak of the CUDA cores: SMs x 128 FP32 lanes x 2 flop x clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def batched_bytes(info, precision, R):
    """Algorithmic bytes of one batched step: A streamed once (values, 16-bit
    codes, FP16 row scales) plus every right-hand side's state read and
    written once."""
    vb = {"fp32": 4, "fp64": 8, "fp16": 2}[precision]
    sb = 8 if precision == "fp64" else 4
    b = info.nnz_stored * (vb + 2) + 2 * info.n_states * R * sb
    if precision == "fp16":
        b += info.n_states * 4
    return b


def batched_roofline(flops, nbytes, ms, fma_peak, hbm_peak, kernel, tensor_peak=None):
    """Roofline of the batched step on the method's work: 2 x nnz x R flops
    (one multiply-add per nonzero and right-hand side) and its algorithmic
    bytes.  The binding roof is the slower of the FP32 CUDA-core FMA roof and
    the HBM roof; frac = that roof's time / the measured time."""
    t_fma = flops / (fma_peak * 1e12)
    t_hbm = nbytes / (hbm_peak * 1e9)
    t = ms * 1e-3
    if t_fma >= t_hbm:
        out = {"bound": "alu", "achieved": round(flops / t / 1e12, 2), "peak": round(fma_peak, 1),
               "unit": "TFLOP/s", "frac": round(t_fma / t, 4)}
    else:
        out = {"bound": "hbm", "achieved": round(nbytes / t / 1e9, 1), "peak": hbm_peak,
               "unit": "GB/s", "frac": round(t_hbm / t, 4)}
    out.update({"traffic": None, "flops_per_step": flops, "algorithmic_bytes_per_step": int(nbytes),
                "fma_roof_ms": round(t_fma * 1e3, 3), "hbm_roof_ms": round(t_hbm * 1e3, 3),
                "hbm_frac": round(t_hbm / t, 4), "fma_frac": round(t_fma / t, 4),
                "peak_kind": "FP32 FMA derived from the device's SM count and maximum clock; "
                             "HBM measured copy"})
    if kernel == "tensor" and tensor_peak:
        out["tensor_frac_method_flops"] = round(flops / t / 1e12 / tensor_peak, 5)
    return out


def batched_launches(args, tune, info, R):
    """Kernels launched in the timed region of the batched run: per step the
    detector readout (when there are patches), the ledger reduction and the
    product (one launch per tile of right-hand sides, one for the
    shared-memory-halo order and the tensor-core form)."""
    per = (1 if info.n_patch > 0 else 0) + 1
    if args.batched_kernel == "tensor":
        return (per + 1) * args.steps
    if tune is None:
        return None
    if tune["variant"] == 2:
        per += 1
    else:
        per += -(-R // tune["rhs_tile"])
    return per * args.steps


def measure_batched(args, workload_name, precision, R, kernel, steps, warmup, autotune,
                    sim_steps, check=True, local=0):
    """Batched step of R right-hand sides sharing A, timed with CUDA events;
    the plain single-right-hand-side step of the same problem timed on the
    same GPU; sampled per-right-hand-side parity of one more step."""
    import copy
    import numpy as np
    import torch
    from paper_1611_08536_gb300 import drts
    stream = torch.cuda.current_stream()
    prob, srcs = workload(workload_name, precision, R)
    prob.batched_kernel = 1 if kernel == "tensor" else 0
    ctx = drts.Context(prob, max_steps=warmup + steps + 2, stream=stream.cuda_stream)
    for r, sr in enumerate(srcs):
        ctx.set_source(r, sr)
    if args.variant >= 0 or args.threads or args.blocks_per_sm or args.rhs_tile:
        ctx.set_launch(args.blocks_per_sm, args.threads, args.rhs_tile, args.variant)
    tune = ctx.autotune(autotune) if autotune else None
    info = ctx.info()
    ctx.step_n(warmup)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        ctx.step_n(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    parity = None
    if check:
        # one more step from the current states (the delta sources are
        # zero by now), checked row by row in FP64 on sampled planes
        import oracle
        rs = sorted({0, R // 2, R - 1})
        xs = {r: ctx.read_state(r) for r in rs}
        ctx.step_n(1)
        ys = {r: ctx.read_state(r) for r in rs}
        nz = prob.shape[2]
        planes = sorted({0, nz // 2, nz - 1})
        worst = 0.0
        for z in planes:
            c = oracle.assemble(prob, z, z + 1)
            for r in rs:
                yo = oracle.spmv(c, xs[r])
                den = np.abs(yo).sum()
                if den > 0:
                    worst = max(worst, float(np.abs(ys[r][c.row0:c.row0 + c.n_rows] - yo).sum() / den))
        parity = {"planes": planes, "rhs": rs, "rel_l1_one_step": worst}
    ctx.close()
    # the plain per-simulation step of the same problem
    p1 = copy.copy(prob)
    p1.n_rhs = 1
    p1.batched_kernel = 0
    c1 = drts.Context(p1, max_steps=warmup + steps, stream=stream.cuda_stream)
    c1.set_source(0, srcs[0])
    if autotune:
        c1.autotune(autotune)
    c1.step_n(warmup)
    torch.cuda.synchronize()
    ev0.record(stream)
    c1.step_n(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms1 = ev0.elapsed_time(ev1) / steps
    c1.close()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz, mhz_src = sm_max_mhz()
    hbm, _ = peaks()
    tensor_peak = None
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        tensor_peak = json.load(open(pk)).get("bf16_tflops")
    flops = 2.0 * info.nnz * R
    nbytes = batched_bytes(info, precision, R)
    roof = batched_roofline(flops, nbytes, ms, fp32_fma_peak_tflops(sms, mhz), hbm, kernel, tensor_peak)
    roof["peak_kind"] += f" ({sms} SMs, {mhz:.0f} MHz from {mhz_src})"
    return {
        "workload": workload_name, "rhs": R, "grid": list(prob.shape), "nnz": int(info.nnz),
        "precision": precision, "batched_kernel": kernel, "launch": tune,
        "ms_per_step": round(ms, 4), "nnz_rhs_per_s": round(info.nnz * R / (ms * 1e-3) / 1e9, 2),
        "sims_per_s": round(R / (sim_steps * ms * 1e-3), 4),
        "plain_single_rhs_ms_per_step": round(ms1, 4),
        "plain_sims_per_s": round(1.0 / (sim_steps * ms1 * 1e-3), 4),
        "speedup_vs_plain_per_simulation": round(R * ms1 / ms, 2),
        "sim_steps": sim_steps, "roofline": roof, "sampled_parity": parity,
        "gpu_launches": batched_launches(types_ns(batched_kernel=kernel, steps=steps), tune, info, R),
        "clocks": clk.summary(),
    }


def types_ns(**kw):
    import types
    return types.SimpleNamespace(**kw)


def run_batched(args):
    """Batched step: one pass over A serves R right-hand sides.  Reports
    nonzero-RHS products per second, simulations per second for a run of
    --sim-steps steps, and the plain single-RHS step of the same problem
    timed on the same GPU."""
    import torch
    from paper_1611_08536_gb300 import build
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    m = measure_batched(args, args.workload, args.precision, args.rhs, args.batched_kernel, args.steps,
                        args.warmup, args.autotune, args.sim_steps, check=args.check, local=local)
    line = {
        "metric": "DRTS batched step, nonzero x right-hand-side products per second",
        "value": m["nnz_rhs_per_s"], "unit": "G nnz-rhs/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f16-matrix/f32-state"}[args.precision],
        "data": "synthetic",
        "config": {k: m[k] for k in ("workload", "rhs", "grid", "nnz", "batched_kernel", "precision",
                                     "launch", "sims_per_s", "plain_single_rhs_ms_per_step",
                                     "plain_sims_per_s", "speedup_vs_plain_per_simulation",
                                     "sim_steps")},
        "roofline": m["roofline"], "sampled_parity": m["sampled_parity"],
        "gpu_launches": m["gpu_launches"], "clocks": m["clocks"],
    }
    print(json.dumps(line), flush=True)


def measure_served(args, n_requests, rate, step_scale, resident, tick_steps, streams, policy_name,
                   baselines="run", local=0):
    """Served stream: seeded Poisson arrivals submitted in real time to the
    continuous-batching server; sims/s and p50/p99 latency, next to the same
    requests run without the server.  baselines = "run" runs every request
    alone and every source as its own single-rhs simulation, one after
    another; "estimate" times the single-rhs step once per grid side and
    multiplies out (for requests with their full step counts, whose plain
    runs would take minutes); "none" skips both."""
    import copy
    import numpy as np
    import torch
    from paper_1611_08536_gb300 import drts
    from paper_1611_08536_gb300 import inputs as I
    stream = I.served_stream(n_requests, rate, seed=4)
    for r in stream:
        r.n_steps = max(1, int(round(r.n_steps * step_scale)))
    lat, queue = [], []
    tick_host = []
    policy = drts.SERVE_SHORTEST_FIRST if policy_name == "shortest" else drts.SERVE_FIFO
    with drts.Server(max_resident=resident, steps_per_tick=tick_steps, n_streams=streams,
                     policy=policy) as srv:
        t0 = time.perf_counter()
        ids, pending = [], list(stream)
        with ClockSampler(local) as clk:
            while pending or len(ids) == 0 or srv.stats()["completed"] + srv.stats()["failed"] < len(stream):
                now = time.perf_counter() - t0
                while pending and pending[0].arrival_s <= now:
                    r = pending.pop(0)
                    ids.append(srv.submit(r.problem, r.sources, r.n_steps))
                st = srv.stats()
                if st["resident"] == 0 and st["queued"] == 0 and pending:
                    time.sleep(min(0.01, max(0.0, pending[0].arrival_s - now)))
                    continue
                tt = time.perf_counter()
                srv.tick()
                tick_host.append(time.perf_counter() - tt)
        makespan = time.perf_counter() - t0
        for rid in ids:
            inf = srv.poll(rid)
            lat.append(inf.latency_s)
            queue.append(inf.queue_s)
        stats = srv.stats()
    n = len(stream)
    n_sims = sum(len(r.sources) for r in stream)
    out = {
        "workload": "served_stream", "requests": n, "simulations": n_sims,
        "arrival_rate_per_s": rate, "step_scale": step_scale,
        "steps": [r.n_steps for r in stream], "sides": [r.problem.shape[0] for r in stream],
        "sources": [len(r.sources) for r in stream],
        "max_resident": resident, "steps_per_tick": tick_steps, "streams": streams,
        "policy": policy_name,
        "requests_per_s": round(n / makespan, 4), "sims_per_s": round(n_sims / makespan, 4),
        "latency_s": {"p50": round(float(np.percentile(lat, 50)), 3),
                      "p99": round(float(np.percentile(lat, 99)), 3),
                      "max": round(float(np.max(lat)), 3)},
        "queue_s": {"p50": round(float(np.percentile(queue, 50)), 3),
                    "p99": round(float(np.percentile(queue, 99)), 3)},
        "makespan_s": round(makespan, 3),
        "tick_wall_s": {"n": len(tick_host), "p50": round(float(np.percentile(tick_host, 50)), 5)
                        if tick_host else None},
        "server_stats": stats,
        "tick_graph_host_ms": {
            "updated_in_place": round(1e3 * (stats["host_graph_s"] - stats["host_instantiate_s"])
                                      / max(stats["graph_updates"], 1), 4),
            "instantiated": round(1e3 * stats["host_instantiate_s"] / max(stats["graph_instantiations"], 1), 4),
            "updates": stats["graph_updates"], "instantiations": stats["graph_instantiations"],
            "note": "host time to capture the tick's launches and update the kept executable graph, against "
                    "capture + instantiate (what every tick paid when each tick instantiated its graph)"},
        "clocks": clk.summary(),
    }
    if baselines == "run":
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for r in stream:
            with drts.Context(r.problem, max_steps=r.n_steps) as ctx:
                for q, sr in enumerate(r.sources):
                    ctx.inject_source(q, sr.state, sr.weight, r.sources[0].t0, r.sources[0].profile)
                ctx.step_n(r.n_steps)
                ctx.read_detectors(0)
        seq = time.perf_counter() - t1
        t2 = time.perf_counter()
        for r in stream:
            p1 = copy.copy(r.problem)
            p1.n_rhs = 1
            for sr in r.sources:
                with drts.Context(p1, max_steps=r.n_steps) as ctx:
                    ctx.inject_source(0, sr.state, sr.weight, r.sources[0].t0, r.sources[0].profile)
                    ctx.step_n(r.n_steps)
                    ctx.read_detectors(0)
        plain = time.perf_counter() - t2
        out["sequential_requests"] = {"requests_per_s": round(n / seq, 4), "seconds": round(seq, 3),
                                      "note": "each request alone, its sources batched"}
        out["plain_per_simulation"] = {"simulations": n_sims, "seconds": round(plain, 3),
                                       "sims_per_s": round(n_sims / plain, 4),
                                       "note": "every source a separate single-rhs run, one after another"}
        out["speedup_vs_plain_per_simulation"] = round(plain / makespan, 3)
    elif baselines == "estimate":
        # single-rhs step time of each grid side (the requests' own media
        # differ only in values, not in the matrix size), times steps x sources
        ms_side = {}
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cs = torch.cuda.current_stream()
        for r in stream:
            side = r.problem.shape[0]
            if side in ms_side:
                continue
            p1 = copy.copy(r.problem)
            p1.n_rhs = 1
            with drts.Context(p1, max_steps=40, stream=cs.cuda_stream) as ctx:
                ctx.inject_source(0, r.sources[0].state, r.sources[0].weight, r.sources[0].t0,
                                  r.sources[0].profile)
                ctx.autotune(2)
                ctx.step_n(5)
                torch.cuda.synchronize()
                ev0.record(cs)
                ctx.step_n(30)
                ev1.record(cs)
                torch.cuda.synchronize()
                ms_side[side] = ev0.elapsed_time(ev1) / 30
        plain = sum(ms_side[r.problem.shape[0]] * 1e-3 * r.n_steps * len(r.sources) for r in stream)
        out["plain_per_simulation"] = {
            "simulations": n_sims, "seconds_estimated": round(plain, 3),
            "sims_per_s": round(n_sims / plain, 4),
            "single_rhs_ms_per_step_by_side": {str(k): round(v, 4) for k, v in sorted(ms_side.items())},
            "note": "every source as its own single-rhs simulation, one after another: the measured "
                    "single-rhs step time of each grid side x steps x sources"}
        out["speedup_vs_plain_per_simulation"] = round(plain / makespan, 3)
    return out


def run_serve(args):
    """Served stream as its own benchmark line (see measure_served)."""
    import torch
    from paper_1611_08536_gb300 import build
    torch.cuda.set_device(0)
    build.build()
    m = measure_served(args, args.serve_requests, args.serve_rate, args.serve_step_scale,
                       args.serve_resident, args.serve_tick_steps, args.serve_streams, args.serve_policy,
                       baselines=("estimate" if args.serve_estimate_baselines
                                  else "run" if args.serve_baselines else "none"))
    line = {
        "metric": "DRTS served stream: simulations per second (continuous batching)",
        "value": m["sims_per_s"], "unit": "sims/s", "n_gpus": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {k: m[k] for k in ("workload", "requests", "simulations", "arrival_rate_per_s",
                                     "step_scale", "max_resident", "steps_per_tick", "streams",
                                     "policy")},
    }
    line.update({k: v for k, v in m.items() if k not in line["config"]})
    print(json.dumps(line), flush=True)


def run_reference(args):
    import numpy as np
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    prob, _ = workload(args.workload, args.precision)
    z = prob.shape[2] // 2
    c = oracle.assemble(prob, z, z + 1)
    x = np.random.default_rng(0).random(prob.n_states)
    threads = oracle.max_threads()
    for _ in range(args.warmup):
        oracle.spmv(c, x, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.spmv(c, x, threads)
    dt = time.perf_counter() - t0
    v = round(c.nnz * args.steps / dt / 1e9, 4)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(prob.shape),
                   "sample": f"rows of z-plane {z} ({c.nnz} nnz) per step"},
        "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": threads,
                         "sample": f"FP64 CSR SpMV over z-plane {z} of the workload per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_functionals(args):
    """Cost of the Eq. 26/27 extensions on the headline workload: the plain
    step, then with --point-detectors sparse detector rows (16 states each),
    then also with a sub-step source (the Gaussian pulse split over the dr/c
    sub-intervals of each step)."""
    import numpy as np
    import torch
    from paper_1611_08536_gb300 import build, drts
    from paper_1611_08536_gb300 import inputs as I
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    prob, src = workload(args.workload, args.precision)
    total = 3 * (args.warmup + args.steps) + 1
    ctx = drts.Context(prob, max_steps=total, stream=stream.cuda_stream)
    ctx.set_source(0, src)
    tune = ctx.autotune(args.autotune) if args.autotune else None
    info = ctx.info()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed():
        ctx.step_n(args.warmup)
        torch.cuda.synchronize()
        ev0.record(stream)
        ctx.step_n(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / args.steps

    with ClockSampler(local) as clk:
        ms_plain = timed()
        # point detectors: 4x4 blocks of +z states on the middle plane
        nx, ny, nz = prob.shape
        n_det = args.point_detectors
        det, st = [], []
        dz = I.direction_index(0, 0, 1)
        for d in range(n_det):
            bx, by = (d * 4) % (nx - 4), ((d * 4) // (nx - 4) * 4) % (ny - 4)
            for q in range(16):
                det.append(d)
                st.append(prob.state(bx + q % 4, by + q // 4, nz // 2, dz))
        ctx.set_point_detectors(n_det, det, st, np.ones(len(st)))
        ms_point = timed()
        n_sub = ctx.substep_count(int(src.state[0]))
        prof = np.repeat(src.profile[:, None] / n_sub, n_sub, 1)
        ctx.inject_source_substeps(0, src.state, src.weight, src.t0, prof)
        ms_both = timed()
    ctx.close()
    line = {
        "metric": "DRTS step with point detectors and sub-step sources (overhead vs plain step)",
        "value": round(100.0 * (ms_both / ms_plain - 1.0), 2), "unit": "% of the plain step",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_both, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f16-matrix/f32-state"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, "nnz": int(info.nnz), "launch": tune,
                   "point_detectors": n_det, "point_entries": len(st), "substeps": int(n_sub),
                   "ms_plain": round(ms_plain, 4), "ms_point_detectors": round(ms_point, 4),
                   "ms_point_and_substep": round(ms_both, 4),
                   "gnnz_per_s_plain": round(info.nnz / (ms_plain * 1e-3) / 1e9, 1)},
        # per step: point detectors, product, sub-step sources
        "gpu_launches": 3 * args.steps, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="drts", choices=["drts", "reference"])
    ap.add_argument("--workload", default="three_layers_128",
                    help="<generator>_<size> or config:<name of a JSON problem file>")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--variant", type=int, default=-1)
    ap.add_argument("--autotune", type=int, default=2, help="timed steps per candidate (0 = off)")
    ap.add_argument("--rhs", type=int, default=1, help="right-hand sides (batched step when > 1)")
    ap.add_argument("--rhs-tile", type=int, default=0, help="batched: right-hand sides per pass (0 = default)")
    ap.add_argument("--step-mode", default="launch", choices=["launch", "persistent"])
    ap.add_argument("--serve", action="store_true", help="served-stream benchmark")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-step-scale", type=float, default=0.1)
    ap.add_argument("--serve-resident", type=int, default=16)
    ap.add_argument("--serve-tick-steps", type=int, default=20)
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--serve-policy", default="fifo", choices=["fifo", "shortest"],
                    help="admission order of queued requests")
    ap.add_argument("--no-serve-baselines", dest="serve_baselines", action="store_false",
                    help="skip the one-after-another and per-simulation baseline runs")
    ap.add_argument("--serve-estimate-baselines", action="store_true",
                    help="estimate the per-simulation baseline from the single-rhs step timed once per "
                         "grid side (for requests with their full step counts)")
    ap.add_argument("--sim-steps", type=int, default=1500, help="steps per simulation for sims/s")
    ap.add_argument("--batched-kernel", default="tensor", choices=["cuda", "tensor"],
                    help="batched product: tcgen05 tensor-core form (default) or CUDA-core form")
    ap.add_argument("--functionals", action="store_true",
                    help="cost of point detectors and sub-step sources on the workload")
    ap.add_argument("--point-detectors", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-check", dest="check", action="store_false")
    ap.add_argument("--sub", default="fp16,batched,fcc,served",
                    help="sub-lines of the default run (comma list of fp16, batched, fcc, served; '' = none)")
    ap.add_argument("--sub-fcc-box", default="192x160x160",
                    help="close-packed box (nx x ny x nz lattice units, nx even) of the fcc sub-line")
    ap.add_argument("--sub-batched-workload", default="inclusions_96")
    ap.add_argument("--sub-batched-steps", type=int, default=10)
    ap.add_argument("--sub-served-requests", type=int, default=7)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    args.sub = [x for x in args.sub.split(",") if x]
    if args.impl == "reference":
        run_reference(args)
    elif args.serve:
        run_serve(args)
    elif args.functionals:
        run_functionals(args)
    elif args.rhs > 1:
        run_batched(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
