"""Benchmark: contraction TFLOP/s and amplitudes/s of random-circuit amplitudes on GB300.

Workload (default): a seeded 7x7 random circuit of depth 1+32+1 (sqrt(X), sqrt(Y), T
single-qubit gates, CZs over 8 nearest-neighbour patterns; bond dimension 16 per edge),
complex64, 6 open output sites -> 64 amplitudes per x1 batch (fast sampling, Sec. III.B),
no cuts (largest intermediate 2^32 elements = 32 GiB), plain FP32 SIMT path.  One step =
one x1 batch through the whole path: fold, scale, 48 contraction steps, FP64 sum.
Counted work is Eq. 1 (F = 8 sqrt(v0 v1 v2) per contraction), 2.256e14 flop per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl qfx|reference]
                  [--workload full|small|kstep|batch|batch_small|permute|adjoint|sample|wide|region]

The default line also carries, each with its own clock record and roofline: every
split-precision mode on the same workload (precision_modes), the adjoint at 6x6x(1+24+1)
(adjoint), the permute kernel against HBM bandwidth (permute), a 128-item subset of the
uneven-shape batch mix (batch: one persistent launch vs per-item launches, FP32 and
BF16x3), the FP64 oracle on the host cores (cpu_baseline) and, last, a compact summary of
all of them.  Workloads other than full/small print their own JSON line: kstep (the
dominant step's kernel in one precision), batch / batch_small (the full 512-item mix or
4096 small items), permute, adjoint, sample (fast sampling with frugal rejection, ideal
and at a quarter of the paths), wide (slices of the 121-qubit 11x11x(1+24+1) shape),
region (slices of contraction-tree plans for 7x7x(1+40+1) and 8x8x(1+32+1)).

Multi-GPU (torchrun): replicas -- each rank contracts its own x1 batches (no exchange on
the data path); value is the sum over ranks, time the max over ranks ("weak" scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rqc_inputs as ri  # noqa: E402

METRIC = "contraction TFLOP/s & amplitudes/s at rel err<=1e-5; % of tensor/HBM roofline"
WORKLOADS = {
    "full": dict(rows=7, cols=7, depth=32, n_open=6, seed=0),
    "small": dict(rows=7, cols=7, depth=24, n_open=6, seed=0),   # profiling case (128 MiB boundary)
}
# DRAM bytes (read + write) per launch of the dominant kernel: dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of the same kernel on the kernel case
# (K = N = 256, 2^18 columns: 1.0290e9 B), scaled by the columns of a full launch
# (2^24 / 2^18 = 64); the traffic grows in proportion to the columns (B read once, C
# written once).
TRAFFIC = {"full": 1.0290e9 * 64, "small": None}


def workload_desc(w):
    return (f"{w['rows']}x{w['cols']}x(1+{w['depth']}+1) RQC seed {w['seed']}, complex64, "
            f"|x2|={w['n_open']} -> {1 << w['n_open']} amplitudes per x1 batch, no cuts, FP32 SIMT")


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_median": statistics.median(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- helpers
def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part", "processor\t: 0")) and ":" in ln:
                    v = ln.split(":", 1)[1].strip()
                    if v and not v.isdigit():
                        return v
    except OSError:
        pass
    return platform.machine()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def blas_threads():
    """Threads of the BLAS numpy calls (threadpoolctl when installed, else the OpenBLAS
    default, one per core)."""
    try:
        from threadpoolctl import threadpool_info
        n = [i["num_threads"] for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(n[0])
    except ImportError:
        pass
    return int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))


# Eq. 1 work of one x1 batch (|x2| = 6) of 7x7x(1+24+1), seed 0, in the line-sweep plan
# (qfx_plan_info's flops_per_item; tests/test_abi_host.py checks the value): the unit the
# full-route CPU figure is counted in.
FLOPS_7x7x24 = 226265202688.0
OPEN_7x7 = [13, 20, 27, 34, 41, 48]    # the planner's six open sites on a 7x7 grid


def cpu_full_route():
    """The oracle as it stands, end to end: oracle.network.amplitudes_open (time fold,
    row-major sweep of np.tensordot in complex128, BLAS on every core) on one x1 batch of
    7x7x(1+24+1) -- the largest shape of the benchmark's family the oracle finishes uncut
    in seconds (7x7x(1+32+1) needs 2^32 complex128 values per tensor and more host memory
    than the benchmark host has)."""
    from oracle import network
    circ = ri.rqc(7, 7, 24, seed=0)
    x1 = int(ri.random_bitstrings(49, 1, seed=1000)[0])
    t0 = time.perf_counter()
    network.amplitudes_open(circ, x1, OPEN_7x7)
    dt = time.perf_counter() - t0
    return {"value": FLOPS_7x7x24 / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(),
            "blas_threads": blas_threads(), "kind": "oracle",
            "sample": f"oracle.network.amplitudes_open, one x1 batch (64 amplitudes) of "
                      f"7x7x(1+24+1) in {dt:.1f} s; Eq. 1 flops of that batch / time; host "
                      f"{cpu_model()}", "amplitudes_per_s": 64.0 / dt, "seconds": dt}


def cpu_step_sample(seconds: float = 4.0, cols: int = 1 << 16):
    """The oracle's contraction routine (oracle.network.contract_network: labelled
    np.tensordot, BLAS threads) on a bounded sample of the benchmark's dominant step,
    K = N = 256 (two bond legs of 4 bits each), `cols` of its 2^24 columns, repeated for
    about `seconds`.  Returns (TFLOP/s, repetitions, seconds)."""
    from oracle import network
    K = N = 256
    S = ri.random_complex((16, 16, 16, 16), seed=1).astype(np.complex128)      # [up][left][right][down]
    B = ri.random_complex((cols, 16, 16), seed=2).astype(np.complex128)         # [s][v][h]
    sl = ["u", "l", "r", "d"]
    bl = ["s", "u", "l"]
    flops = 8.0 * K * N * cols
    t0 = time.perf_counter()
    reps = 0
    while True:
        network.contract_network([(B, bl), (S, sl)])
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return flops * reps / dt / 1e12, reps, dt


def shared_config(w):
    """The config object both arms print for the default workload."""
    return {"workload": workload_desc(w), "grid": [w["rows"], w["cols"]], "depth": w["depth"],
            "n_open": w["n_open"], "l2": "inputs larger than L2 (each big step reads and writes 32 GiB)",
            "precision": "fp32_simt"}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 oracle on the host cores: each step is the oracle's contraction routine on a
    bounded sample (2^16 of 2^24 columns) of the workload's dominant step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    times, tf = [], []
    reps_total = 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rate, reps, dt = cpu_step_sample(seconds=1.0)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
            tf.append(rate)
            reps_total += reps
    value = float(np.mean(tf))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic", "config": shared_config(w),
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": os.cpu_count(),
                         "blas_threads": blas_threads(), "kind": "oracle",
                         "sample": f"oracle.network.contract_network (np.tensordot, complex128) on "
                                   f"2^16 of the 2^24 columns of the dominant step (K = N = 256), "
                                   f"{reps_total} contractions over {args.steps} steps of ~1 s; "
                                   f"host {cpu_model()}"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def fp32_peak(torch, dev, sm_max):
    """FP32 FMA-pipe peak, TFLOP/s: SMs x 128 lanes x 2 flop x clock (recipe unit counts)."""
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    return n_sm * 128 * 2 * sm_max * 1e6 / 1e12, n_sm


def run_qfx(args):
    import torch
    import torch.distributed as dist
    world, rank, local = dist_env()
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1905_00444_gb300 as qfx

    w = WORKLOADS[args.workload]
    circ = ri.rqc(w["rows"], w["cols"], w["depth"], seed=w["seed"])
    t0 = time.perf_counter()
    plan = qfx.Plan(qfx.Circuit(circ), n_open=w["n_open"])
    plan.upload()
    plan_s = time.perf_counter() - t0
    flops_step = plan.stats["flops_per_item"] * plan.n_slices
    amps_step = 1 << w["n_open"]
    nq = w["rows"] * w["cols"]
    total = args.warmup + args.steps
    x1_host = ri.random_bitstrings(nq, total * world, seed=1000)[rank * total:(rank + 1) * total]
    x1_dev = torch.tensor(x1_host.view(np.int64), device=dev)
    ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device=dev)
    out = torch.empty((1, amps_step), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for i in range(args.warmup):
        qfx.amplitudes(plan, x1_dev[i:i + 1], workspace=ws, out=out, stream=stream)
    barrier()

    # ---- device-timed region: inputs resident in HBM -------------------------------
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    clocks = ClockSampler(f"GPU-{uuid}" if uuid is not None else str(local))
    clocks.start()
    qfx.profile_enable(True)
    launches0 = qfx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for i in range(args.warmup, total):
        qfx.amplitudes(plan, x1_dev[i:i + 1], workspace=ws, out=out, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = qfx.launch_count() - launches0
    qfx.profile_enable(False)
    recs = qfx.profile_collect()
    clk = clocks.stop()
    amax = torch.tensor([elapsed], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(amax, op=dist.ReduceOp.MAX)
    elapsed = float(amax.item())

    # ---- end to end through the public API with host buffers ----------------------
    e2e_steps = min(args.steps, 5)
    pin_x1 = torch.tensor(x1_host.view(np.int64)).pin_memory()
    pin_out = torch.empty((1, amps_step), dtype=torch.complex128).pin_memory()
    barrier()
    e0 = time.perf_counter()
    for i in range(args.warmup, args.warmup + e2e_steps):
        d = pin_x1[i:i + 1].to(dev, non_blocking=True)
        qfx.amplitudes(plan, d, workspace=ws, out=out, stream=stream)
        pin_out.copy_(out, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
    e_el = time.perf_counter() - e0
    emax = torch.tensor([e_el], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(emax, op=dist.ReduceOp.MAX)
    e_el = float(emax.item())

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel (largest contraction step) ---------------
    big = plan.steps[plan.stats["largest_step"]]
    dom = [r for r in recs if r["kind"] == 0 and r["flops"] == big["flops"]]
    dom_ms = float(np.mean([r["ms"] for r in dom])) if dom else float("nan")
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak, n_sm = fp32_peak(torch, dev, sm_max)
    achieved = big["flops"] / (dom_ms / 1e3) / 1e12
    kern_total = sum(r["ms"] for r in recs)
    share = {}
    for r in recs:
        key = {0: "contraction_step", 1: "fold", 4: "permute"}.get(r["kind"], str(r["kind"]))
        share[key] = share.get(key, 0.0) + r["ms"]

    value = flops_step * args.steps * world / elapsed / 1e12
    cfg = shared_config(w)
    cfg.update({"n_slices": plan.n_slices, "flops_per_step": flops_step,
                "max_intermediate_bytes": plan.stats["max_elements"] * 8, "plan_s": plan_s})
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
        "data": "synthetic", "config": cfg,
        "amplitudes_per_s": amps_step * args.steps * world / elapsed,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": TRAFFIC.get(args.workload),
                     "kernel": f"cgemm_step variant {big['variant']} (P,K,N,Sd)="
                               f"({big['P']},{big['K']},{big['N']},{big['Sd']})",
                     "launches_timed": len(dom),
                     "peak_note": f"{n_sm} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz"},
        "kernel_share": {k: v / kern_total for k, v in share.items()} if kern_total else {},
        "e2e": {"value": flops_step * e2e_steps * world / e_el / 1e12, "unit": "TFLOP/s",
                "amplitudes_per_s": amps_step * e2e_steps * world / e_el, "steps": e2e_steps,
                "h2d_bytes_per_step": 8, "d2h_bytes_per_step": 16 * amps_step},
        "clocks": clk,
        "gpu_launches": int(launches),
    }
    sub_steps = max(1, min(args.steps, 5))
    sub_warm = max(1, min(args.warmup, 2))
    if not args.no_modes and world == 1:
        line["precision_modes"] = {m: run_mode(qfx, torch, circ, w, m, x1_dev, sub_steps, sub_warm,
                                               dev, stream)
                                   for m in ("bf16x3", "tf32x3", "bf16x2", "bf16x3_fast")}
    del ws
    torch.cuda.empty_cache()
    if not args.no_configs and world == 1:
        line["adjoint"] = measure_adjoint(qfx, torch, steps=sub_steps, warmup=sub_warm)
        line["permute"] = measure_permute(qfx, torch, steps=sub_steps, warmup=sub_warm)
        line["batch"] = measure_batch(qfx, torch, BATCH_MIX_SUBSET, 8, steps=1, warmup=1,
                                      tc=True, autotune=not args.no_autotune)
        line["region"] = {"workload": "7x7x(1+40+1) RQC seed 0, contraction-tree plan at an 8 GiB cap, "
                                      "|x2| = 6, BF16x3, seeded slices of one x1 batch",
                          **region_entry(qfx, torch, qfx.Circuit(ri.rqc(7, 7, 40, seed=0)), "bf16x3",
                                         steps=2, warmup=1, dev=dev)}
    if world == 1 and not args.no_cpu:
        cpu = cpu_full_route()
        rate, reps, dt = cpu_step_sample(seconds=4.0)
        cpu["step_sample"] = {"value": rate, "unit": "TFLOP/s",
                              "what": f"oracle.network.contract_network on 2^16 of the 2^24 columns "
                                      f"of the dominant step, {reps} reps in {dt:.1f} s"}
        line["cpu_baseline"] = cpu
    line["summary"] = summarize(line)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _r(x, nd=3):
    return None if x is None else float(f"{x:.{nd}g}")


def summarize(line):
    """Compact figures of every part of the line, printed last (the end of the line is
    what a truncated log keeps)."""
    s = {"fp32": {"tflops": _r(line["value"]), "frac": _r(line["roofline"]["frac"]),
                  "e2e": _r(line["e2e"]["value"]), "mhz": line["clocks"].get("sm_mhz")}}
    for m, d in line.get("precision_modes", {}).items():
        s[m] = {"tflops": _r(d["value"]), "frac_probe": _r(d["roofline"]["tensor_probe"]["frac"]),
                "err_vs_fp32": _r(d["max_rel_diff_vs_fp32"], 2), "mhz": d["clocks"].get("sm_mhz")}
    if "adjoint" in line:
        a = line["adjoint"]
        s["adjoint"] = {"fwd_ms": _r(a["forward_ms"]), "bwd_ms": _r(a["backward_ms"]),
                        "bwd_frac": _r(a["roofline"]["frac"]), "graph_ms": _r(a["graph_forward_backward_ms"])}
    if "permute" in line:
        s["permute_frac"] = [_r(c["frac"], 2) for c in line["permute"]["cases"]]
    if "batch" in line:
        b = line["batch"]
        s["batch_tflops"] = {"persistent": _r(b["fp32_persistent"]["value"]),
                             "per_item": _r(b["fp32_per_item"]["value"]),
                             "bf16x3_graph": _r(b["bf16x3_graph"]["value"]) if b.get("bf16x3_graph") else None,
                             "bf16x3_per_item": _r(b["bf16x3_per_item"]["value"]) if b.get("bf16x3_per_item") else None}
    if "region" in line:
        g = line["region"]
        s["region_7x7x40_bf16x3"] = {"tflops": _r(g["value"]), "frac_probe": _r(g["roofline"]["tensor_probe"]["frac"]),
                                     "amps_per_s_f0.006": _r(g["amplitudes_per_s_at_fidelity_0.006"])}
    if "cpu_baseline" in line:
        c = line["cpu_baseline"]
        s["cpu"] = {"tflops": _r(c["value"]), "cores": c["cores"],
                    "step_sample": _r(c["step_sample"]["value"])}
    return s


# Tensor-pipe work per counted complex multiply-add (8 counted flops): 4 real products,
# each the sum of 6 (BF16x3) or 3 (TF32x3, BF16x2) term products -> 48 or 24 flops of the
# mode's type.  TF32 runs at half the BF16 rate (nominal ratio).
TENSOR_FACTOR = {"bf16x3": 48 / 8, "tf32x3": 24 / 8, "bf16x2": 24 / 8}
TENSOR_PEAK_RATIO = {"bf16x3": 1.0, "tf32x3": 0.5, "bf16x2": 1.0}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0}, "fallback"


def run_mode(qfx, torch, circ, w, mode, x1_dev, steps, warmup, dev, stream):
    """The same workload with the contraction steps on tcgen05 in a split precision, and
    the largest per-amplitude difference to the FP32 path (floor 2^(-n/2))."""
    fast = mode.endswith("_fast")
    mode = mode.replace("_fast", "")
    plan32 = qfx.Plan(qfx.Circuit(circ), n_open=w["n_open"])
    plan = qfx.Plan(qfx.Circuit(circ), n_open=w["n_open"], precision=mode, fast_accumulation=fast)
    plan.upload()
    ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device=dev)
    out = torch.empty((1, 1 << w["n_open"]), dtype=torch.complex128, device=dev)
    for i in range(warmup):
        qfx.amplitudes(plan, x1_dev[i:i + 1], workspace=ws, out=out, stream=stream)
    torch.cuda.synchronize(dev)
    qfx.profile_enable(True)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(warmup, warmup + steps):
        qfx.amplitudes(plan, x1_dev[i:i + 1], workspace=ws, out=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    qfx.sync()
    qfx.profile_enable(False)
    recs = qfx.profile_collect()
    el = e0.elapsed_time(e1) / 1e3
    got = out.clone()
    ref = qfx.amplitudes(plan32, x1_dev[warmup + steps - 1:warmup + steps], workspace=ws, stream=stream)
    qfx.sync()
    floor = 2.0 ** (-w["rows"] * w["cols"] / 2)
    diff = float((torch.abs(got - ref) / torch.clamp(torch.abs(ref), min=floor)).max())
    del ws
    flops = plan.stats["flops_per_item"] * plan.n_slices
    big = plan.steps[plan.stats["largest_step"]]
    dom = [r["ms"] for r in recs if r["kind"] == 0 and r["flops"] == big["flops"]]
    dom_ms = float(np.mean(dom)) if dom else float("nan")
    counted = big["flops"] / (dom_ms / 1e3) / 1e12
    peaks, src = measured_peaks()
    peak = peaks["bf16_tflops_sustained"] * TENSOR_PEAK_RATIO[mode]
    burst = peaks["bf16_tflops"] * TENSOR_PEAK_RATIO[mode]
    achieved = counted * TENSOR_FACTOR[mode]
    probe = qfx.tensor_peak(mode, 1 << 16)   # this kind's MMA rate, measured here
    return {"value": flops * steps / el / 1e12, "unit": "TFLOP/s",
            "amplitudes_per_s": (1 << w["n_open"]) * steps / el,
            "ms_per_step": 1e3 * el / steps, "steps": steps,
            "largest_step_counted_tflops": counted, "max_rel_diff_vs_fp32": diff,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "frac_of_burst": achieved / burst, "traffic": None,
                         "tensor_probe": {"tflops": probe, "frac": achieved / probe},
                         "peak_source": f"{src} bf16 sustained x {TENSOR_PEAK_RATIO[mode]}; tensor-pipe "
                                        f"flops = {TENSOR_FACTOR[mode]:g} x counted"},
            "clocks": clk}


def measure_adjoint(qfx, torch, steps, warmup):
    """6x6x(1+24+1) parametrised RQC, 128 bitstrings, L = sum |amp|^2: forward amplitudes
    and the adjoint's gradients of every gate tensor (every step output stored), CUDA
    events; backward work model = 3 forward-equivalents (forward, reverse step, site-
    gradient GEMM)."""
    circ = ri.rqc(6, 6, 24, seed=0, parametrised=True)
    x1 = torch.tensor(ri.random_bitstrings(36, 1, seed=9).view(np.int64), device="cuda")
    out = torch.empty((1, 128), dtype=torch.complex128, device="cuda")
    plan = qfx.Plan(qfx.Circuit(circ), n_open=7)
    ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device="cuda")
    bws = torch.empty(plan.backward_workspace_bytes(), dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        amp = qfx.amplitudes(plan, x1, workspace=ws, out=out)
        qfx.amplitudes_backward(plan, x1, 2 * amp, workspace=bws)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    f_ms, b_ms = [], []
    for _ in range(max(steps, 60)):      # ~0.3 s, so the clock record has samples
        ev[0].record()
        amp = qfx.amplitudes(plan, x1, workspace=ws, out=out)
        ev[1].record()
        qfx.amplitudes_backward(plan, x1, 2 * amp, workspace=bws)
        ev[2].record()
        torch.cuda.synchronize()
        f_ms.append(ev[0].elapsed_time(ev[1]))
        b_ms.append(ev[1].elapsed_time(ev[2]))
    clk = clocks.stop()
    qfx.sync()
    # the same forward + backward replayed from one CUDA graph (no launch gaps)
    gs = torch.cuda.Stream()
    with torch.cuda.stream(gs):
        amp = qfx.amplitudes(plan, x1, workspace=ws, out=out)
        qfx.amplitudes_backward(plan, x1, 2 * amp, workspace=bws)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        amp = qfx.amplitudes(plan, x1, workspace=ws, out=out)
        qfx.amplitudes_backward(plan, x1, 2 * amp, workspace=bws)
    with torch.cuda.stream(gs):
        graph.replay()
        torch.cuda.synchronize()
        ev[0].record(gs)
        for _ in range(50):
            graph.replay()
        ev[1].record(gs)
    torch.cuda.synchronize()
    qfx.sync()
    graph_ms = ev[0].elapsed_time(ev[1]) / 50
    del graph
    flops = plan.stats["flops_per_item"]
    fwd, bwd = float(np.median(f_ms)), float(np.median(b_ms))
    peak, _ = fp32_peak(torch, torch.device("cuda", 0), clk.get("sm_max_mhz") or 2070.0)
    bt = 3 * flops / (bwd / 1e3) / 1e12
    return {"workload": f"6x6x(1+24+1) parametrised RQC, 128 bitstrings, {len(circ.gates)} gate "
                        f"tensors, every step output stored",
            "forward_ms": fwd, "backward_ms": bwd, "forward_tflops": flops / (fwd / 1e3) / 1e12,
            "backward_tflops": bt, "graph_forward_backward_ms": graph_ms,
            "graph_tflops": 4 * flops / (graph_ms / 1e3) / 1e12,
            "roofline": {"bound": "alu", "achieved": bt, "peak": peak, "unit": "TFLOP/s",
                         "frac": bt / peak, "what": "backward, 3 x forward flops / time, FP32 FMA peak"},
            "clocks": clk}


def measure_permute(qfx, torch, steps, warmup):
    """qfx_permute on 2^28-element complex64 tensors (2 GiB in, 2 GiB out): HBM bandwidth
    (16 B per element) against the measured copy bandwidth."""
    peaks, src = measured_peaks()
    out = []
    clocks = ClockSampler(0)
    clocks.start()
    for shape, perm in PERMUTES:
        n = int(np.prod(shape))
        x = torch.randn(n, dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        for _ in range(warmup):
            qfx.permute(x, shape, perm, out=y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(steps, 100)           # ~0.1 s per case, so the clock record has samples
        e0.record()
        for _ in range(reps):
            qfx.permute(x, shape, perm, out=y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = 16.0 * n / (ms / 1e3) / 1e9
        out.append({"shape": list(shape), "perm": list(perm), "ms": ms, "GB/s": gbs,
                    "frac": gbs / peaks["hbm_gbs"]})
        del x, y
    clk = clocks.stop()
    qfx.sync()
    return {"workload": "permute, 2^28 complex64 elements", "roofline": {
        "bound": "hbm", "peak": peaks["hbm_gbs"], "unit": "GB/s", "peak_source": src},
        "cases": out, "clocks": clk}


# ----------------------------------------------------------------------------- batch case
BATCH_MIX_SMALL = [  # many tiny items: launch overhead dominates per-item execution
    (4, 4, 16, 1 << 30, 2048, "x1"),
    (4, 5, 16, 1 << 30, 1024, "x1"),
    (5, 5, 24, 1 << 30, 1024, "x1"),
]
BATCH_MIX = [  # (rows, cols, depth, per-item cap bytes, items, kind)
    (6, 6, 24, 1 << 30, 171, "x1"),       # bond dim 2^3, whole item per x1
    (7, 7, 32, 1 << 30, 171, "slice"),    # 2^4, seeded sample of slices (path subsampling)
    (8, 8, 32, 2 << 30, 166, "slice"),    # 2^4; the line sweep needs a 2 GiB cap (2^57 slices)
    (7, 7, 40, 8 << 30, 4, "slice"),      # 2^5; an 8 GiB cap (2^59 slices), 4.6e13 flop each
]


BATCH_MIX_SUBSET = [  # a quarter of BATCH_MIX, same proportions (the default line's batch)
    (6, 6, 24, 1 << 30, 43, "x1"),
    (7, 7, 32, 1 << 30, 43, "slice"),
    (8, 8, 32, 2 << 30, 41, "slice"),
    (7, 7, 40, 8 << 30, 1, "slice"),
]


def measure_batch(qfx, torch, mix, n_open, steps, warmup, tc, autotune):
    """Work items of uneven shapes from mixed grids: one persistent launch replayed from a
    CUDA graph vs one qfx_amplitudes call per item; with tc, the same items with BF16x3
    plans as one batch (a CUDA graph of per-item launch sequences over parallel lanes) and
    per item.  Results of the batched and per-item runs must be bit-identical."""
    dev = torch.device("cuda", 0)
    items, flops = [], 0.0
    rng = np.random.default_rng(7)
    cache = os.path.join("/tmp", "qfx_autotune_batch.json")
    tc_plan, nq = {}, []   # split-precision twin of each plan; qubits per item
    for (r, c, d, cap, count, kind) in mix:
        n0 = len(items)
        circ = qfx.Circuit(ri.rqc(r, c, d, seed=r * 10 + d))
        plan = qfx.Plan(circ, n_open=n_open, max_intermediate_bytes=cap)
        if autotune:
            qfx.autotune(plan, cache)
            plan = qfx.Plan(circ, n_open=n_open, max_intermediate_bytes=cap, autotune_cache=cache)
        if kind == "x1":
            xs = ri.random_bitstrings(r * c, count, seed=r + d)
            for x in xs:
                items.append((plan, torch.tensor(np.array([x], dtype=np.uint64).view(np.int64), device=dev), 0, 1))
        else:
            x1 = torch.tensor(ri.random_bitstrings(r * c, 1, seed=r + d).view(np.int64), device=dev)
            for sl in sorted(set(int(v) for v in rng.integers(0, plan.n_slices, size=count))):
                items.append((plan, x1, sl, sl + 1))
        flops += plan.stats["flops_per_item"] * (len(items) - n0)
        if tc:
            tp = qfx.Plan(circ, n_open=n_open, max_intermediate_bytes=cap, precision="bf16x3")
            if autotune:   # tensor cores or FP32 tiles, per step shape, by timing
                qfx.autotune(tp, cache)
                tp = qfx.Plan(circ, n_open=n_open, max_intermediate_bytes=cap, precision="bf16x3",
                              autotune_cache=cache)
            tc_plan[id(plan)] = tp
        nq += [r * c] * (len(items) - n0)
    # slots hold the largest item; keep the batch workspace under ~96 GiB
    block = max(p.workspace_bytes(1) for p, _, _, _ in items)
    slots = int(max(2, min(16, (96 << 30) // block)))
    clocks = ClockSampler(0)
    clocks.start()
    batch = qfx.Batch(items, slots=slots)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        for _ in range(max(1, warmup)):
            batch.run(stream=stream)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        batch.run(stream=stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):      # replay() launches on the current stream
        e0.record(stream)
        for _ in range(steps):
            graph.replay()
        e1.record(stream)
    torch.cuda.synchronize(dev)
    qfx.sync()
    t_graph = e0.elapsed_time(e1) / 1e3 / steps
    ref = [o.clone() for o in batch.outs]
    n_tasks_fp32, slots_fp32 = batch.n_tasks, batch.slots
    del graph, batch
    torch.cuda.empty_cache()
    # per-item launches on one shared workspace
    ws = torch.empty(max(p.workspace_bytes(1) for p, _, _, _ in items), dtype=torch.uint8, device=dev)
    outs = [torch.empty_like(o) for o in ref]
    for _ in range(max(1, warmup)):
        for (plan, x1, sb, se), o in zip(items, outs):
            qfx.amplitudes(plan, x1, slice_begin=sb, slice_end=se, workspace=ws, out=o)
    torch.cuda.synchronize(dev)
    l1 = qfx.launch_count()
    e0.record()
    for _ in range(steps):
        for (plan, x1, sb, se), o in zip(items, outs):
            qfx.amplitudes(plan, x1, slice_begin=sb, slice_end=se, workspace=ws, out=o)
    e1.record()
    torch.cuda.synchronize(dev)
    t_items = e0.elapsed_time(e1) / 1e3 / steps
    per_item_launches = (qfx.launch_count() - l1) // steps
    same = all(torch.equal(a, b) for a, b in zip(ref, outs))
    res = {"n_items": len(items), "flops_per_batch": flops,
           "fp32_persistent": {"value": flops / t_graph / 1e12, "ms_per_batch": 1e3 * t_graph,
                               "items_per_s": len(items) / t_graph, "tasks_or_graph_nodes": n_tasks_fp32,
                               "slots": slots_fp32,
                               "what": "one batch replayed from a CUDA graph: items with steps of "
                                       ">= 512 tiles as their own launches, the others in one "
                                       "persistent launch"},
           "fp32_per_item": {"value": flops / t_items / 1e12, "ms_per_batch": 1e3 * t_items,
                             "items_per_s": len(items) / t_items, "kernel_launches": per_item_launches},
           "fp32_identical": bool(same), "autotuned": bool(autotune)}
    del ws
    torch.cuda.empty_cache()
    if tc:
        tc_items = [(tc_plan[id(p)], x1, sb, se) for p, x1, sb, se in items]
        ws_tc = torch.empty(max(p.workspace_bytes(1) for p, _, _, _ in tc_items), dtype=torch.uint8, device=dev)
        outs_tc = [torch.empty_like(o) for o in ref]
        for _ in range(max(1, warmup)):
            for (plan, x1, sb, se), o in zip(tc_items, outs_tc):
                qfx.amplitudes(plan, x1, slice_begin=sb, slice_end=se, workspace=ws_tc, out=o)
        torch.cuda.synchronize(dev)
        e0.record()
        for _ in range(steps):
            for (plan, x1, sb, se), o in zip(tc_items, outs_tc):
                qfx.amplitudes(plan, x1, slice_begin=sb, slice_end=se, workspace=ws_tc, out=o)
        e1.record()
        torch.cuda.synchronize(dev)
        qfx.sync()
        t_tc = e0.elapsed_time(e1) / 1e3 / steps
        worst = 0.0
        for a, b, n in zip(outs_tc, ref, nq):
            fl = 2.0 ** (-n / 2)
            worst = max(worst, float((torch.abs(a - b) / torch.clamp(torch.abs(b), min=fl)).max()))
        del ws_tc
        torch.cuda.empty_cache()
        lane = max(p.workspace_bytes(1) for p, _, _, _ in tc_items)
        gb = qfx.Batch(tc_items, slots=int(max(1, min(16, (96 << 30) // lane))))
        with torch.cuda.stream(stream):
            for _ in range(max(1, warmup)):
                gb.run(stream=stream)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(steps):
                gb.run(stream=stream)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        qfx.sync()
        t_gb = e0.elapsed_time(e1) / 1e3 / steps
        same_tc = all(torch.equal(a, b) for a, b in zip(gb.outs, outs_tc))
        res["bf16x3_per_item"] = {"value": flops / t_tc / 1e12, "ms_per_batch": 1e3 * t_tc}
        res["bf16x3_graph"] = {"value": flops / t_gb / 1e12, "ms_per_batch": 1e3 * t_gb,
                               "lanes": gb.slots, "graph_nodes": gb.n_tasks,
                               "what": "one CUDA graph: items with tensor-core steps (and large "
                                       "ones) as launch sequences over parallel lanes, items "
                                       "whose steps all take FP32 tiles in one persistent "
                                       "launch beside them"}
        res["bf16x3_identical"] = bool(same_tc)
        res["bf16x3_max_rel_diff_vs_fp32"] = worst
        del gb
        torch.cuda.empty_cache()
    res["clocks"] = clocks.stop()
    return res


def run_batch(args):
    """The 512-item mix (batch) or 4096 small items (batch_small); |x2| = 8 (256 amplitudes
    per item) or 4.  The 512-item mix costs ~1.4e15 flop per batch, so it times at most 2
    batches after 1 warm-up."""
    import torch
    import paper_1905_00444_gb300 as qfx
    big = args.workload == "batch"
    mix = BATCH_MIX if big else BATCH_MIX_SMALL
    steps, warmup = (min(args.steps, 2), 1) if big else (args.steps, args.warmup)
    res = measure_batch(qfx, torch, mix, 8 if big else 4, steps, warmup, tc=True,
                        autotune=not args.no_autotune)
    desc = ("batch of 512 work items: 171 x 6x6x(1+24+1) x1 batches (bond dim 2^3); sampled "
            "slices: 171 of 7x7x(1+32+1) (1 GiB cap), 166 of 8x8x(1+32+1) (2 GiB cap), both "
            "bond dim 2^4, and 4 of 7x7x(1+40+1) (8 GiB cap, bond dim 2^5); |x2| = 8") if big else (
            "batch of 4096 small work items: 2048 x 4x4x(1+16+1), 1024 x 4x5x(1+16+1), "
            "1024 x 5x5x(1+24+1) x1 batches; |x2| = 4; FP32 plans and their BF16x3 twins")
    print(json.dumps({"workload": desc, "metric": "contraction TFLOP/s", "unit": "TFLOP/s", **res}),
          flush=True)
    return 0


# ----------------------------------------------------------------------------- adjoint case
def run_adjoint(args):
    """6x6x(1+24+1) circuit with parametrised single-qubit gates, 128 bitstrings
    (|x2| = 7), L = sum |amp|^2: forward amplitudes and the adjoint's gradients for every
    gate tensor, timed separately with CUDA events; the backward both with every step output
    stored (the default at this size) and with one checkpoint per line."""
    import torch
    import paper_1905_00444_gb300 as qfx
    circ = ri.rqc(6, 6, 24, seed=0, parametrised=True)
    x1 = torch.tensor(ri.random_bitstrings(36, 1, seed=9).view(np.int64), device="cuda")
    out = torch.empty((1, 128), dtype=torch.complex128, device="cuda")
    res = {}
    for mode, store, model in (("stored_outputs", 0, 3), ("line_checkpoints", 1, 4)):
        plan = qfx.Plan(qfx.Circuit(circ), n_open=7, adjoint_store_bytes=store)
        ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device="cuda")
        bws = torch.empty(plan.backward_workspace_bytes(), dtype=torch.uint8, device="cuda")
        for _ in range(args.warmup):
            amp = qfx.amplitudes(plan, x1, workspace=ws, out=out)
            g = qfx.amplitudes_backward(plan, x1, 2 * amp, workspace=bws)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        f_ms, b_ms = [], []
        for _ in range(args.steps):
            ev[0].record()
            amp = qfx.amplitudes(plan, x1, workspace=ws, out=out)
            ev[1].record()
            g = qfx.amplitudes_backward(plan, x1, 2 * amp, workspace=bws)
            ev[2].record()
            torch.cuda.synchronize()
            f_ms.append(ev[0].elapsed_time(ev[1]))
            b_ms.append(ev[1].elapsed_time(ev[2]))
        qfx.sync()
        flops = plan.stats["flops_per_item"]
        res[mode] = {"forward_ms": float(np.median(f_ms)), "backward_ms": float(np.median(b_ms)),
                     "forward_tflops": flops / (np.median(f_ms) / 1e3) / 1e12,
                     "backward_model_flops": model * flops,
                     "backward_tflops": model * flops / (np.median(b_ms) / 1e3) / 1e12,
                     "backward_workspace_bytes": plan.backward_workspace_bytes(),
                     "grad_norm": float(torch.linalg.vector_norm(g).item())}
        del ws, bws
    print(json.dumps({
        "workload": "adjoint: 6x6x(1+24+1) parametrised RQC, 128 bitstrings (|x2|=7), "
                    "L = sum |amp|^2, gradients of all %d gate tensors" % len(circ.gates),
        **res,
        "note": "backward work model, in units of the forward's flops: stored outputs = one "
                "forward + a reverse step + a site-gradient GEMM per step (3); line "
                "checkpoints add the line-by-line recompute (4)"}), flush=True)
    return 0


# ----------------------------------------------------------------------------- sampling case
def run_sample(args):
    """Fast sampling with frugal rejection (Sec. III.B) on a 6x6x(1+24+1) RQC, |x2| = 6
    (64 candidates per x1), 256 x1 batches per step, M = 10: amplitudes of every batch and
    the device-side selection, timed with CUDA events (draws uploaded before timing).
    Ideal: the uncut plan.  Noisy (Sec. III.C): two middle bonds cut to 4 slices each
    (16 paths), a quarter of them summed, M * 1/4.  The linear XEB of both sample sets is
    taken from the ideal amplitudes of the same x1 batches."""
    import torch
    import paper_1905_00444_gb300 as qfx
    rows, cols, depth, n_open, nb, M = 6, 6, 24, 6, 256, 10.0
    n = rows * cols
    circ = qfx.Circuit(ri.rqc(rows, cols, depth, seed=0))
    x1s, masks, u = ri.sampling_draws(n, n_open, nb, seed=31)
    x1 = torch.from_numpy(x1s.view(np.int64)).cuda()
    mk = torch.from_numpy(masks.view(np.int64)).cuda()
    ud = torch.from_numpy(u).cuda()

    def leg(plan, slices, m):
        items = nb * (slices[1] - slices[0])
        ws = torch.empty(plan.workspace_bytes(min(items, 64)), dtype=torch.uint8, device="cuda")
        for _ in range(args.warmup):
            qfx.frugal_sample(plan, x1, ud, mk, m, slice_begin=slices[0], slice_end=slices[1],
                              workspace=ws)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ms = []
        for _ in range(args.steps):
            ev[0].record()
            x2, bits, amps = qfx.frugal_sample(plan, x1, ud, mk, m, slice_begin=slices[0],
                                               slice_end=slices[1], workspace=ws)
            ev[1].record()
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        qfx.sync()
        del ws
        t = float(np.median(ms)) / 1e3
        flops = plan.stats["flops_per_item"] * items
        return x2.cpu().numpy(), amps, t, flops

    ideal = qfx.Plan(circ, n_open=n_open)
    x2_i, amps_i, t_i, f_i = leg(ideal, (0, 1), M)
    p_i = (amps_i.abs() ** 2).cpu().numpy()
    cut = qfx.Plan(circ, n_open=n_open, cuts=[(14, 20, 2), (15, 21, 2)])
    q = cut.n_slices // 4
    x2_n, amps_n, t_n, f_n = leg(cut, (0, q), M * 0.25)
    norm_ratio = float((amps_n.abs() ** 2).sum().item() / p_i.sum())

    def xeb(x2):
        ok = x2 >= 0
        return float(2.0 ** n * p_i[np.arange(nb)[ok], x2[ok]].mean() - 1.0), int(ok.sum())

    xi, si = xeb(x2_i)
    xn, sn = xeb(x2_n)
    print(json.dumps({
        "workload": "fast sampling: 6x6x(1+24+1) RQC seed 0, |x2| = 6 (64 candidates per x1), "
                    "256 x1 batches per step, frugal rejection M = 10, FP32 SIMT contraction",
        "ideal": {"samples_per_s": si / t_i, "amplitudes_per_s": nb * 64 / t_i,
                  "ms_per_step": 1e3 * t_i, "tflops": f_i / t_i / 1e12, "samples": si,
                  "acceptance": si / nb, "xeb": xi},
        "noisy_quarter_of_paths": {
            "samples_per_s": sn / t_n, "ms_per_step": 1e3 * t_n, "tflops": f_n / t_n / 1e12,
            "slices": [0, q], "of_slices": cut.n_slices, "norm_ratio": norm_ratio,
            "samples": sn, "xeb": xn},
        "note": "xeb = N mean p(x) - 1 with p from the ideal amplitudes of the same x1 batches "
                "(about 1 for ideal samples, about the path fraction for noisy ones). The line "
                "sweep needs no cut on this grid and the two cuts lower the per-slice work only "
                "from 1.84e10 to 1.52e10 flop, so the quarter of 16 paths costs more than the "
                "ideal run; the path fraction pays where memory forces cuts anyway."}),
        flush=True)
    return 0


# ----------------------------------------------------------------------------- permute case
PERMUTES = [  # (shape, perm): bond-tensor transposes of the kind region plans need
    ((16,) * 7, (6, 5, 4, 3, 2, 1, 0)),           # full reversal: tiled transpose path
    ((256, 256, 256, 16), (0, 2, 1, 3)),          # inner axis kept: row-copy path
    ((4096, 65536), (1, 0)),                      # matrix transpose
    ((16, 16, 16, 16, 16, 16, 16), (0, 1, 3, 2, 4, 6, 5)),
]


def run_permute(args):
    import torch
    import paper_1905_00444_gb300 as qfx
    print(json.dumps(measure_permute(qfx, torch, args.steps, args.warmup)), flush=True)
    return 0


# ----------------------------------------------------------------------------- 121 qubits
def run_wide(args):
    """The paper's 11x11x(1+24+1) shape (121 qubits, two-word bitstrings, mean |amp|^2 =
    2^-121) under a 64 GiB cap on the largest intermediate: 2^31 slices (paths, Sec. III.A)
    of 2.5e14 flop each.  Each timed step contracts one seeded slice of one x1 batch
    (|x2| = 6), in FP32 and in BF16x3; the slice sum of a fraction f of the paths gives
    amplitudes of fidelity about f (Sec. III.C)."""
    import torch
    import paper_1905_00444_gb300 as qfx
    dev = torch.device("cuda", 0)
    circ = qfx.Circuit(ri.rqc(11, 11, 24, seed=0))
    words = ri.random_bitstring_words(121, 1, seed=11)
    x1 = torch.tensor(words.view(np.int64), device=dev)
    peaks, src = measured_peaks()
    res = {}
    for fam, cap, prec in (("line", 64 << 30, "fp32"), ("line", 64 << 30, "bf16x3"),
                           ("tree", 32 << 30, "fp32"), ("tree", 32 << 30, "bf16x3")):
        plan = qfx.Plan(circ, n_open=6, max_intermediate_bytes=cap, precision=prec, family=fam)
        plan.upload()
        sids = [int(v) for v in np.random.default_rng(3).integers(0, plan.n_slices, args.warmup + args.steps)]
        ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device=dev)
        out = torch.empty((1, 64), dtype=torch.complex128, device=dev)
        for s in sids[:args.warmup]:
            qfx.amplitudes(plan, x1, slice_begin=s, slice_end=s + 1, workspace=ws, out=out)
        torch.cuda.synchronize(dev)
        clocks = ClockSampler(0)
        clocks.start()
        qfx.profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for s in sids[args.warmup:]:
            qfx.amplitudes(plan, x1, slice_begin=s, slice_end=s + 1, workspace=ws, out=out)
        e1.record()
        torch.cuda.synchronize(dev)
        qfx.profile_enable(False)
        recs = qfx.profile_collect()
        clk = clocks.stop()
        qfx.sync()
        el = e0.elapsed_time(e1) / 1e3
        flops = plan.stats["flops_per_item"]
        big = plan.steps[plan.stats["largest_step"]]
        dom = [r["ms"] for r in recs if r["kind"] == 0 and r["flops"] == big["flops"]]
        counted = big["flops"] / (float(np.mean(dom)) / 1e3) / 1e12 if dom else float("nan")
        if prec == "fp32":
            peak, _ = fp32_peak(torch, dev, clk.get("sm_max_mhz") or 2070.0)
            roof = {"bound": "alu", "achieved": counted, "peak": peak, "unit": "TFLOP/s",
                    "frac": counted / peak}
        else:
            probe = qfx.tensor_peak("bf16x3", 1 << 16)
            roof = {"bound": "tensor", "achieved": counted * TENSOR_FACTOR["bf16x3"], "unit": "TFLOP/s",
                    "peak": peaks["bf16_tflops"], "frac_of_burst": counted * TENSOR_FACTOR["bf16x3"] / peaks["bf16_tflops"],
                    "tensor_probe": {"tflops": probe, "frac": counted * TENSOR_FACTOR["bf16x3"] / probe}}
        res[f"{fam}_{prec}"] = {"value": flops * args.steps / el / 1e12, "unit": "TFLOP/s",
                     "ms_per_slice": 1e3 * el / args.steps, "timed_slices": args.steps,
                     "slices": plan.n_slices, "flops_per_slice": flops, "cap_bytes": cap,
                     "seconds_per_x1_batch": plan.n_slices * el / args.steps,
                     "dominant_step": f"(P,K,N,Sd)=({big['P']},{big['K']},{big['N']},{big['Sd']})",
                     "roofline": roof, "clocks": clk}
        del ws
        torch.cuda.empty_cache()
    print(json.dumps({"workload": "11x11x(1+24+1) RQC seed 0 (121 qubits), |x2| = 6: line sweep at a "
                                  "64 GiB cap and tree plan at a 32 GiB cap; one seeded slice per step",
                      "metric": "contraction TFLOP/s", **res}), flush=True)
    return 0


# ----------------------------------------------------------------------------- region plans
def region_entry(qfx, torch, circ, prec, steps, warmup, dev):
    """One tree plan at an 8 GiB cap, |x2| = 6: `steps` seeded slices of one x1 batch timed
    with CUDA events after `warmup` others, with the largest node's roofline, kernel shares
    and the amplitude rates at the paper's fidelity (0.6%) and at full fidelity."""
    n = circ.rows * circ.cols
    x1 = torch.tensor(ri.random_bitstrings(n, 1, seed=2).view(np.int64), device=dev)
    t0 = time.perf_counter()
    plan = qfx.Plan(circ, n_open=6, max_intermediate_bytes=8 << 30, family="tree", precision=prec)
    plan_s = time.perf_counter() - t0
    sids = [int(v) for v in np.random.default_rng(1).integers(0, plan.n_slices, warmup + steps)]
    ws = torch.empty(plan.workspace_bytes(1), dtype=torch.uint8, device=dev)
    out = torch.empty((1, 64), dtype=torch.complex128, device=dev)
    for s in sids[:warmup]:
        qfx.amplitudes(plan, x1, slice_begin=s, slice_end=s + 1, workspace=ws, out=out)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    qfx.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for s in sids[warmup:]:
        qfx.amplitudes(plan, x1, slice_begin=s, slice_end=s + 1, workspace=ws, out=out)
    e1.record()
    torch.cuda.synchronize(dev)
    qfx.profile_enable(False)
    recs = qfx.profile_collect()
    clk = clocks.stop()
    qfx.sync()
    el = e0.elapsed_time(e1) / 1e3
    flops = plan.stats["flops_per_item"]
    kt = {}
    for r in recs:
        k = {0: "contraction_step", 1: "fold", 4: "permute"}.get(r["kind"], str(r["kind"]))
        kt[k] = kt.get(k, 0.0) + r["ms"]
    tot = sum(kt.values()) or 1.0
    big = plan.steps[plan.stats["largest_step"]]
    dom = [r["ms"] for r in recs if r["kind"] == 0 and r["step"] == plan.stats["largest_step"]]
    dom_tf = big["flops"] / (float(np.mean(dom)) / 1e3) / 1e12 if dom else float("nan")
    if prec == "fp32":
        peak, _ = fp32_peak(torch, dev, clk.get("sm_max_mhz") or 2070.0)
        roof = {"bound": "alu", "achieved": dom_tf, "peak": peak, "unit": "TFLOP/s", "frac": dom_tf / peak}
    else:
        probe = qfx.tensor_peak("bf16x3", 1 << 16)
        ach = dom_tf * TENSOR_FACTOR["bf16x3"]
        roof = {"bound": "tensor", "achieved": ach, "unit": "TFLOP/s",
                "tensor_probe": {"tflops": probe, "frac": ach / probe}}
    roof["kernel"] = f"largest node (P,K,N,Sd)=({big['P']},{big['K']},{big['N']},{big['Sd']})"
    spl = el / steps
    f_paper = 0.006          # the paper's fidelity for 7x7x(1+40+1) (Sec. V, Table I)
    res = {
        "value": flops * steps / el / 1e12, "unit": "TFLOP/s", "ms_per_slice": 1e3 * spl,
        "amplitudes_per_s_at_fidelity_0.006": 64.0 / (max(1, round(f_paper * plan.n_slices)) * spl),
        "amplitudes_per_s_full": 64.0 / (plan.n_slices * spl),
        "slices": plan.n_slices, "flops_per_slice": flops, "flops_per_x1_batch": flops * plan.n_slices,
        "max_intermediate_bytes": plan.stats["max_elements"] * 8, "workspace_bytes": plan.workspace_bytes(1),
        "plan_s": plan_s, "cuts": len(plan.cuts), "kernel_share": {k: v / tot for k, v in kt.items()},
        "roofline": roof, "clocks": clk}
    del ws
    torch.cuda.empty_cache()
    return res


def run_region(args):
    """Region (contraction-tree) plans for the paper's 7x7x(1+40+1) shape and for
    8x8x(1+32+1), both at an 8 GiB cap on the largest intermediate, |x2| = 6: each timed
    step contracts one seeded slice of one x1 batch, in FP32 and in BF16x3, against the line
    sweep's slice count and work at the same cap (planned only)."""
    import torch
    import paper_1905_00444_gb300 as qfx
    dev = torch.device("cuda", 0)
    res = {}
    for rows, cols, depth in ((7, 7, 40), (8, 8, 32)):
        circ = qfx.Circuit(ri.rqc(rows, cols, depth, seed=0))
        line = qfx.Plan(circ, n_open=6, max_intermediate_bytes=8 << 30)
        entry = {prec: region_entry(qfx, torch, circ, prec, args.steps, args.warmup, dev)
                 for prec in ("fp32", "bf16x3")}
        entry["line_sweep_at_same_cap"] = {"slices": line.n_slices, "flops_per_slice": line.stats["flops_per_item"],
                                           "flops_per_x1_batch": line.stats["flops_per_item"] * line.n_slices}
        res[f"{rows}x{cols}x(1+{depth}+1)"] = entry
    print(json.dumps({"workload": "region (contraction-tree) plans at an 8 GiB cap, |x2| = 6, "
                                  "one seeded slice per step", "metric": "contraction TFLOP/s", **res}),
          flush=True)
    return 0


# ----------------------------------------------------------------------------- kernel case
def run_kstep(args):
    """The dominant contraction step alone (K = N = 256 as in the 7x7x32 interior steps)
    on 2^18 of its 2^24 columns: 512 MiB in, 512 MiB out (larger than L2), the small case
    used for ncu captures of that kernel."""
    import torch
    import paper_1905_00444_gb300 as qfx
    P, K, N, NL, Sd = 1, 256, 256, 256, 1 << 18
    S = torch.from_numpy(ri.random_complex((K * N,), seed=1)).cuda()
    B = torch.from_numpy(ri.random_complex((P * K * Sd,), seed=2)).cuda()
    C = torch.empty(P * N * Sd, dtype=torch.complex64, device="cuda")
    prec = args.precision.replace("_fast", "")
    var = 12 if args.precision.endswith("_fast") else -1
    scratch = torch.empty(max(1, qfx.qfx.step_scratch_bytes(K, N, prec)), dtype=torch.uint8,
                          device="cuda")
    for _ in range(args.warmup):
        qfx.contract_step(S, B, P, K, N, NL, Sd, out=C, precision=prec, scratch=scratch, variant=var)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        qfx.contract_step(S, B, P, K, N, NL, Sd, out=C, precision=prec, scratch=scratch, variant=var)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    flops = 8.0 * P * K * N * Sd
    line = {"workload": "dominant step (P,K,N,Sd)=(1,256,256,2^18)", "precision": args.precision, "ms": ms,
            "tflops": flops / ms / 1e9, "steps": args.steps}
    if args.precision == "fp32":
        # library comparator, run only: cuBLAS complex64 GEMM (torch.matmul, TF32 off) on
        # the same product, C[n][s] = sum_k S[k][n] B[k][s] (P = 1)
        torch.backends.cuda.matmul.allow_tf32 = False
        St, Bm = S.view(K, N).t(), B.view(K, Sd)
        Cm = torch.empty(N, Sd, dtype=torch.complex64, device="cuda")
        for _ in range(args.warmup):
            torch.matmul(St, Bm, out=Cm)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            torch.matmul(St, Bm, out=Cm)
        e1.record()
        torch.cuda.synchronize()
        cms = e0.elapsed_time(e1) / args.steps
        rel = (torch.linalg.vector_norm(Cm.reshape(-1) - C) / torch.linalg.vector_norm(Cm)).item()
        line["cublas_cgemm"] = {"ms": cms, "tflops": flops / cms / 1e9, "rel_diff_to_qfx": rel}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="qfx", choices=["qfx", "reference"])
    ap.add_argument("--workload", default="full",
                    choices=sorted(WORKLOADS) + ["kstep", "batch", "batch_small", "permute", "adjoint",
                                                 "sample", "wide", "region"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16x3", "tf32x3", "bf16x2", "bf16x3_fast"],
                    help="kernel case only; the amplitude run reports every mode")
    ap.add_argument("--no-modes", action="store_true", help="skip the split-precision runs")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the adjoint, permute and batch parts of the default line")
    ap.add_argument("--no-autotune", action="store_true", help="batch case: planner's default tiles")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "kstep":
        return run_kstep(args)
    if args.workload in ("batch", "batch_small"):
        return run_batch(args)
    if args.workload == "permute":
        return run_permute(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "sample":
        return run_sample(args)
    if args.workload == "wide":
        return run_wide(args)
    if args.workload == "region":
        return run_region(args)
    return run_qfx(args)


if __name__ == "__main__":
    sys.exit(main())
