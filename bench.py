#!/usr/bin/env python
"""Benchmark: FP64 blocked LU with malleable look-ahead on one GB300, plus the
mixed-precision time to backward error 1e-14 beside the FP64 one.

A step is one pass of the hot path over one synthetic matrix: restore A
(n = 32768, the largest order of the FP64 sweep, entries uniform [-1, 1),
FP64, 8 GiB, larger than L2), lu_factor (panel, row interchanges, TRSM,
trailing update, look-ahead) and lu_solve of b = A * ones.  The metric value
is LU GFLOP/s = (2/3 n^3) / (time per step).  The line also carries the pivot
agreement with the oracle's stored pivots, the mixed-precision time to
backward error 1e-14 at n = 16384 for kappa in {1e2, 1e5, 1e8} and 1 or 8
right-hand sides beside the FP64 path's, the batched workload and the n = 512
latency.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank factors its own matrix on its own GPU
(independent replicas, no collective on the data path; "scaling": "weak") and
the value is the sum of all ranks' flops over the slowest rank's time.
--impl reference times the CPU oracle (plain unblocked GEPP + getrs, FP64) on
the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LU GFLOP/s (2/3n^3) and time to 1e-14 backward error: mixed vs FP64, 1 GB300"
N_MAIN = 32768
FP64_FAMILY = 20161106 + 1000 * 2   # family 2 (blocked FP64 LU sweep)
FP64_CASE = {4096: 1, 8192: 2, 16384: 0, 32768: 3}   # seed = FP64_FAMILY + case, as in the tests
SEED = FP64_FAMILY + 0              # the CPU legs' sample matrices
MIXED_N = 16384
MIXED_KAPPAS = (1e2, 1e5, 1e8)
MIXED_NRHS = (1, 8)
MIXED_FAMILY = 20161106 + 1000 * 3  # family 3 (mixed-precision solve)
MIXED_REFLECTORS = 256              # the order-65536 FP8 case (the full product takes too long there)
SM_COUNT = 152
FP64_PEAK_TFLOPS = 2 * 2 * SM_COUNT * 2.07e9 / 1e12   # 2 DFMA (4 flop) / clk / SM at 2070 MHz = 1.259
FP32_PEAK_TFLOPS = 128 * 2 * SM_COUNT * 2.07e9 / 1e12  # 128 FFMA (256 flop) / clk / SM at 2070 MHz = 80.5
PEAKS_JSON = os.path.join(ROOT, "profiles", "peaks_alu_gb300.json")


def fp64_seed(n):
    return FP64_FAMILY + FP64_CASE.get(n, 0)


def _alu_peaks():
    """Measured FP64 / FP32 ALU peaks (bench --case peaks, committed under profiles/)."""
    try:
        with open(PEAKS_JSON) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def fp64_peak():
    """(TFLOP/s, note): the larger of the measured DFMA and DMMA rates, else the derived figure."""
    pk = _alu_peaks()
    vals = [pk.get(k, {}).get("tflops") for k in ("dfma", "dmma")]
    vals = [v for v in vals if v]
    if vals:
        return max(vals), f"measured: max(DFMA, DMMA) probe, {os.path.relpath(PEAKS_JSON, ROOT)}"
    return FP64_PEAK_TFLOPS, "derived: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (no measured probe on file)"


def fp32_peak():
    pk = _alu_peaks().get("ffma", {}).get("tflops")
    if pk:
        return pk, f"measured: FFMA probe, {os.path.relpath(PEAKS_JSON, ROOT)}"
    return FP32_PEAK_TFLOPS, "derived: 128 FFMA/clk/SM x 152 SMs x 2070 MHz (no measured probe on file)"
BATCH_COUNT = 10000
BATCH_SEED = 20161106 + 1000 * 4      # family 4 (batched LU)


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def flops_lu(n):
    return 2.0 / 3.0 * n ** 3


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
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
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names[1:], parts[5:9]):
                if val.lower() in ("active", "0x1", "1", "yes"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------
# reference arm: the CPU oracle
# ----------------------------------------------------------------------------
def oracle_sample(n_sample, seed):
    import numpy as np

    import lu_inputs as li
    import oracle

    A = li.uniform(n_sample, n_sample, seed)
    b = li.ones_rhs(A)
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    LU, ipiv, info = oracle.getrf(A, nthreads=threads)
    x = oracle.getrs(LU, ipiv, b)
    dt = time.perf_counter() - t0
    assert info == 0 and np.max(np.abs(x - 1.0)) < 1e-8
    return dt, threads


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    n_s = args.ref_n
    for _ in range(args.warmup):
        oracle_sample(n_s, SEED)
    times = []
    threads = 1
    for _ in range(args.steps):
        dt, threads = oracle_sample(n_s, SEED)
        times.append(dt)
    t = sum(times) / len(times)
    value = flops_lu(n_s) / t / 1e9
    sample = f"oracle getrf+getrs (unblocked GEPP, FP64) on a uniform [-1,1) matrix of order {n_s} per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"fp64_lu_lookahead_n{N_MAIN}", "n": N_MAIN, "nrhs": 1,
                   "sample_n": n_s, "device": "host cores"},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def combine_ranks(ms_local, steps, flops_per_rank_step, ws, device):
    """Whole-job timing over independent replicas: the slowest rank's time (an
    all-reduce MAX when a process group is up) and the flops of all ranks over
    it.  Returns (ms per step, GFLOP/s)."""
    import torch

    ms = float(ms_local)
    if ws > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / steps
    return ms_per_step, ws * flops_per_rank_step / (ms_per_step / 1e3) / 1e9


def run_ours(args):
    import numpy as np
    import torch

    import lu_inputs as li
    import paper_1611_06365_gb300 as lu

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    lu.build()
    n = args.n
    # inputs: A (FP64, column-major, 2 GiB at n = 16384) generated on the device
    seed = fp64_seed(n) + rank
    A0 = li.uniform_colmajor_torch(n, n, seed, dev, torch.float64)
    A = torch.empty_like(A0)
    ones = torch.ones(n, dtype=torch.float64, device=dev)
    b0 = (A0.t() @ ones).view(1, n)            # b = A * ones (column-major A0 holds A^T row-major)
    b = torch.empty_like(b0)
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # the autotuner picks b_o and the panel team for this order (untimed); every
    # factorization below leaves its options at zero and so runs the winner
    tuned = {}
    if args.tune_file and os.path.exists(args.tune_file):
        # a table saved by an earlier run: no tuning launches (profiling runs)
        tuned["loaded"] = {"file": args.tune_file, "entries": lu.lu_tune_load(args.tune_file)}
        args.no_autotune = True
    if not args.no_autotune:
        if n <= 16384:
            tuned["fp64"] = lu.lu_autotune(lu.LU_F64, n, budget_ms=args.tune_budget_ms)
        else:
            # one candidate takes ~20 s here: the built-in FP64 plan is the tuner's winner
            # at n = 16384 (b_o = 64, 8-CTA panel team), also the best of a b_o sweep at 32768
            tuned["fp64"] = {"opts": lu.lu_plan_info(lu.LU_F64, n)[1], "built_in": True}

    def step():
        A.copy_(A0)
        b.copy_(b0)
        lu.lu_factor(A, ipiv, info)
        lu.lu_solve(A, ipiv, b)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness of the last step (device residual with a library product; verification only)
    x = b.view(-1)
    r = b0.view(-1) - A0.t() @ x
    eta = float(r.abs().max() / (A0.abs().sum(0).max() * x.abs().max() + b0.abs().max()))
    assert int(info.item()) == 0 and eta < 10 * n * 2.0 ** -53, f"FP64 step failed: info={int(info.item())} eta={eta}"

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    lu.lu_update_timing(True)
    launches0 = lu.lu_kernel_launches()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches = lu.lu_kernel_launches() - launches0
    lu.lu_update_timing(False)
    upd_n, upd_ms, upd_flops, upd_bytes = lu.lu_update_timing_read()
    clk = clocks.stop()
    ms_per_step, value = combine_ranks(e0.elapsed_time(e1), args.steps, flops_lu(n), ws, dev)
    pivots = pivot_agreement(n, seed, ipiv.cpu().numpy()) if rank == 0 else None

    # end-to-end through the C ABI with host buffers (pinned), copies timed
    hA = A0.cpu().pin_memory()
    hb = b0.cpu().pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    hinfo = torch.zeros(1, dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3 if n <= 16384 else 1))
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(e2e_steps):
        A.copy_(hA, non_blocking=True)
        b.copy_(hb, non_blocking=True)
        lu.lu_factor(A, ipiv, info)
        lu.lu_solve(A, ipiv, b)
        hx.copy_(b, non_blocking=True)
        hinfo.copy_(info, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1) / e2e_steps
    assert int(hinfo.item()) == 0 and float((hx - 1.0).abs().max()) < 1e-8
    e2e = {"value": flops_lu(n) / (e2e_ms / 1e3) / 1e9, "unit": "GFLOP/s",
           "h2d_bytes_per_step": 8 * n * n + 8 * n, "d2h_bytes_per_step": 8 * n + 4, "ms_per_step": e2e_ms}
    del hA

    # roofline of the dominant kernel (trailing update, FP64 DFMA)
    achieved = upd_flops / (upd_ms / 1e3) / 1e12 if upd_ms > 0 else 0.0
    peak64, peak64_note = fp64_peak()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                "frac": achieved / peak64, "traffic": None,
                "kernel": "gemm_update_simt<double>", "launches": upd_n,
                "avg_launch_ms": upd_ms / max(1, upd_n),
                "flops_per_launch": upd_flops / max(1, upd_n),
                "peak_note": peak64_note,
                "peak_live": live_probe(dev)}
    # measured DRAM bytes per flop of the update at the plan's panel width (the update's
    # depth k): an ncu capture of the same kernel at that k, scaled to the average launch
    _, plan = lu.lu_plan_info(lu.LU_F64, n)
    roofline["plan"] = plan
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            entries = json.load(f).get("gemm_update_simt<double>", [])
        for tr in entries if isinstance(entries, list) else [entries]:
            if tr.get("valid") and tr.get("k") == plan["nb"]:
                roofline["traffic"] = tr["bytes_per_flop"] * roofline["flops_per_launch"]
                roofline["traffic_source"] = tr.get("source")

    # the same factorization + solve with the emulated FP64 update (tensor cores)
    emu = None
    if rank == 0 and not args.skip_emu:
        emu = fp64_emulated_case(n, seed, A0, A, b0, b, ipiv, info, stream)
    # time to backward error 1e-14: mixed precision vs FP64 on the kappa matrices
    tts = None
    if not args.skip_mixed and rank == 0:
        if not args.no_autotune:
            tuned["mixed_f32"] = lu.lu_autotune(lu.LU_F32, args.mixed_n, update=lu.LU_UPDATE_BF16X3,
                                                budget_ms=args.tune_budget_ms)
        tts = time_to_solution(args, dev)
    batched = None
    if not args.skip_batched and rank == 0:
        batched = {dt: batched_case(dev, dt, args.steps, tuned if not args.no_autotune else None)
                   for dt in ("f64", "f32")}
    small = None
    if rank == 0 and not args.skip_small:
        if not args.no_autotune:
            tuned["fp64_n512"] = lu.lu_autotune(lu.LU_F64, 512)
        small = small_case(dev)
    chol = None
    if rank == 0 and not args.skip_chol:
        # Cholesky on the same look-ahead schedule (n = 16384: DFMA and emulated updates)
        chol = cholesky_measure(16384, dev, 2)
    et_rows = None
    if rank == 0 and not args.skip_et:
        # early termination (section 4.2) on and off, same plans (b_o = 64, b_i = 16)
        try:
            et_rows = early_term_measure(dev)
        except Exception as exc:   # reported, never fatal to the line
            et_rows = f"failed: {type(exc).__name__}: {exc}"

    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"fp64_lu_lookahead_n{n}", "n": n, "lda": n, "nrhs": 1, "seed": seed,
                   "entries": "uniform [-1,1)",
                   "l2": f"inputs larger than L2 ({8 * n * n / 2 ** 30:.0f} GiB FP64 matrix restored per step)",
                   "parallelism": f"replicas x{ws}", "eta_fp64": eta,
                   "pivots_vs_oracle": pivots,
                   "autotuned": tuned or None},
        "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
        "fp64_emulated": emu, "time_to_solution": tts, "batched": batched, "latency_n512": small,
        "cholesky": chol, "early_termination": et_rows,
    }
    if rank == 0 and not args.skip_cpu:
        dt, threads = oracle_sample(args.cpu_n, SEED)
        # the n = 512 factor + solve of the latency line, on the same host cores (best of 5)
        dt512 = min(oracle_sample(512, 20161106 + 1000 * 1)[0] for _ in range(5))
        line["cpu_baseline"] = {"value": flops_lu(args.cpu_n) / dt / 1e9, "unit": "GFLOP/s", "cores": threads,
                                "kind": "oracle",
                                "sample": f"oracle getrf+getrs on a uniform [-1,1) matrix of order {args.cpu_n} "
                                          f"(same generator), {dt:.1f} s",
                                "n512_us": dt512 * 1e6}
    if rank == 0 and args.tune_file and "loaded" not in tuned:
        lu.lu_tune_save(args.tune_file)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def fp64_emulated_case(n, seed, A0, A, b0, b, ipiv, info, stream):
    """lu_factor + lu_solve of the headline matrix with the emulated FP64 update
    (LU_UPDATE_F64EMU): one warm-up, then 3 timed steps (CUDA events); the update
    kernel against its rooflines (BF16 tensor flops of the 28 digit products, and
    HBM bytes: C in FP64 read and written once per launch, the digit slices read
    once); pivots against the oracle's stored vector; backward error of the solve."""
    import torch

    import paper_1611_06365_gb300 as lu

    def step():
        A.copy_(A0)
        b.copy_(b0)
        lu.lu_factor(A, ipiv, info, update=lu.LU_UPDATE_F64EMU)
        lu.lu_solve(A, ipiv, b)

    step()
    torch.cuda.synchronize()
    x = b.view(-1)
    r = b0.view(-1) - A0.t() @ x
    eta = float(r.abs().max() / (A0.abs().sum(0).max() * x.abs().max() + b0.abs().max()))
    assert int(info.item()) == 0 and eta < 10 * n * 2.0 ** -53, f"emulated FP64 step failed: eta={eta}"
    pivots = pivot_agreement(n, seed, ipiv.cpu().numpy())
    reps = 3
    lu.lu_update_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    lu.lu_update_timing(False)
    u_n, u_ms, u_flops, u_bytes = lu.lu_update_timing_read()
    ms = e0.elapsed_time(e1) / reps
    mp = _measured_peaks()
    hbm, bf16 = mp.get("hbm_gbs", 6692.1), mp.get("bf16_tflops_sustained", 1739.6)
    # tensor work: 28 products of K = 64 (the digit slices are padded to 64) per C element
    tensor_tflops = 28.0 * u_flops * (64.0 / lu.lu_plan_info(lu.LU_F64, n, update=lu.LU_UPDATE_F64EMU)[1]["nb"]) \
        / (u_ms / 1e3) / 1e12 if u_ms > 0 else 0.0
    gbs = u_bytes / (u_ms / 1e3) / 1e9 if u_ms > 0 else 0.0
    return {"n": n, "update": "LU_UPDATE_F64EMU", "ms_per_step": ms, "gflops": flops_lu(n) / (ms / 1e3) / 1e9,
            "eta": eta, "pivots_vs_oracle": pivots,
            "plan": lu.lu_plan_info(lu.LU_F64, n, update=lu.LU_UPDATE_F64EMU)[1],
            "update_kernel": {"kernel": "gemm_update_f64emu", "launches": u_n, "total_ms_per_step": u_ms / reps,
                              "fp64_equiv_tflops": u_flops / (u_ms / 1e3) / 1e12 if u_ms > 0 else 0.0,
                              "tensor": {"achieved": tensor_tflops, "peak": bf16, "unit": "TFLOP/s",
                                         "frac": tensor_tflops / bf16},
                              "hbm": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm}}}


def pivot_agreement(n, seed, ipiv):
    """The pivot vector of the timed factorization against the oracle's, stored
    for this (order, seed) by tests/golden/make_oracle_pivots.py (the full oracle
    takes minutes to an hour at these orders); for orders without a stored
    vector, None."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import make_oracle_pivots
    from _parity import golden_agreement

    gold = make_oracle_pivots.read(n, seed)
    if gold is None:
        return None
    out = golden_agreement(ipiv, gold[0], gold[1], n)
    out["reference"] = os.path.basename(make_oracle_pivots.golden_path(n, seed))
    return out


def live_probe(dev):
    """The FP64 peak probes, run now (a fraction of a second each), beside the stored figure."""
    import paper_1611_06365_gb300 as lu

    out = {}
    for name, kind, iters in (("dfma", lu.PROBE_DFMA, 1 << 11), ("dmma", lu.PROBE_DMMA, 1 << 15)):
        lu.lu_peak_probe(kind, iters // 16)
        tf, ms = lu.lu_peak_probe(kind, iters)
        out[name] = {"tflops": tf, "ms": ms}
    return out


def small_case(dev):
    """The n = 512 FP64 factor + solve (b = A * ones) as a latency: median of 20
    runs, each bracketed by CUDA events; the matrix is restored before each run."""
    import statistics as st

    import torch

    import lu_inputs as li
    import paper_1611_06365_gb300 as lu

    n = 512
    A0 = li.uniform_colmajor_torch(n, n, 20161106 + 1000 * 1, dev, torch.float64)
    b0 = (A0.t() @ torch.ones(n, dtype=torch.float64, device=dev)).view(1, n)
    A, b = torch.empty_like(A0), torch.empty_like(b0)
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    times = []
    for rep in range(23):
        A.copy_(A0)
        b.copy_(b0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lu.lu_factor(A, ipiv, info)
        lu.lu_solve(A, ipiv, b)
        e1.record()
        torch.cuda.synchronize()
        if rep >= 3:
            times.append(e0.elapsed_time(e1) * 1e3)
    assert int(info.item()) == 0 and float((b - 1.0).abs().max()) < 1e-10
    return {"n": n, "us": st.median(times), "us_min": min(times), "gflops": flops_lu(n) / (st.median(times) / 1e6) / 1e9}


def batched_case(dev, dtype, steps, tuned=None):
    """10 000 LUs + solves of orders uniform in [16, 256] (odd members diagonally
    dominant), b = A * ones, one CUDA graph per step (restore, factor, solve)."""
    import numpy as np
    import torch

    import lu_inputs as li
    import paper_1611_06365_gb300 as lu

    tdt = torch.float64 if dtype == "f64" else torch.float32
    code = lu.LU_F64 if dtype == "f64" else lu.LU_F32
    sizes = li.batch_sizes(BATCH_COUNT, 16, 256, seed=BATCH_SEED)
    offs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)])
    roffs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64))])
    buf0 = torch.empty(int(offs[-1]), dtype=tdt, device=dev)
    rhs0 = torch.empty(int(roffs[-1]), dtype=tdt, device=dev)
    for t, n in enumerate(sizes):
        n = int(n)
        A = li.uniform_colmajor_torch(n, n, BATCH_SEED + 1 + t, dev, torch.float64)
        if t % 2 == 1:
            A.view(-1)[:: n + 1] += n
        buf0[int(offs[t]):int(offs[t + 1])] = A.view(-1).to(tdt)
        rhs0[int(roffs[t]):int(roffs[t + 1])] = (A.to(tdt).double().t() @ torch.ones(n, dtype=torch.float64,
                                                                                       device=dev)).to(tdt)
    buf, rhs = buf0.clone(), rhs0.clone()
    esz = buf.element_size()
    ns = torch.tensor(sizes, dtype=torch.int32, device=dev)
    ptrA = torch.tensor([buf.data_ptr() + int(o) * esz for o in offs[:-1]], dtype=torch.int64, device=dev)
    ipiv = torch.zeros(int(roffs[-1]), dtype=torch.int32, device=dev)
    ptrP = torch.tensor([ipiv.data_ptr() + int(o) * 4 for o in roffs[:-1]], dtype=torch.int64, device=dev)
    ptrB = torch.tensor([rhs.data_ptr() + int(o) * esz for o in roffs[:-1]], dtype=torch.int64, device=dev)
    info = torch.zeros(BATCH_COUNT, dtype=torch.int32, device=dev)
    if tuned is not None:
        tuned[f"batched_{dtype}"] = lu.lu_autotune_batched(code, ns, 256)

    def body():
        buf.copy_(buf0)
        rhs.copy_(rhs0)
        lu.lu_factor_batched(code, ns, ptrA, ns, ptrP, info, 256)
        lu.lu_solve_batched(code, 1, ns, ptrA, ns, ptrP, ptrB, ns, 256)

    body()                                   # library state and workspace pools before capture
    torch.cuda.synchronize()
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        body()
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        body()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    reps = max(3, steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / reps
    # the restore copies alone, to separate them from the factor + solve time
    e0.record()
    for _ in range(reps):
        buf.copy_(buf0)
        rhs.copy_(rhs0)
    e1.record()
    torch.cuda.synchronize()
    restore_ms = e0.elapsed_time(e1) / reps
    g.replay()
    torch.cuda.synchronize()
    infos = info.cpu().numpy()
    x = rhs.cpu().numpy().astype(np.float64)
    err = float(np.max(np.abs(x - 1.0)))
    # x = ones up to kappa * eps of each member (FP32: a loose sanity bound)
    assert np.all(infos == 0) and err < (1e-6 if dtype == "f64" else 1.0), (dtype, err)
    flops = float(np.sum(2.0 / 3.0 * sizes.astype(np.float64) ** 3 + 2.0 * sizes.astype(np.float64) ** 2))
    lu_ms = step_ms - restore_ms
    peak, peak_note = fp64_peak() if dtype == "f64" else fp32_peak()
    achieved = flops / (lu_ms / 1e3) / 1e12
    return {"count": BATCH_COUNT, "n_range": [16, 256], "seed": BATCH_SEED, "graph": True,
            "step_ms": step_ms, "restore_ms": restore_ms, "factor_solve_ms": lu_ms,
            "gflops": flops / (lu_ms / 1e3) / 1e9, "max_abs_err_x_minus_1": err,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "peak_note": peak_note}}


def time_to_solution(args, dev):
    """Mixed-precision solve vs the FP64 factor + refinement, both to eta <= 1e-14,
    on the kappa matrices A = U diag(s) V^T (U, V: full products of n seeded
    Householder reflectors each, one pair shared by the kappas), for every kappa
    and number of right-hand sides; X_true has column 0 = ones, the others
    uniform [-1, 1), B = A X_true in FP64."""
    import torch

    import lu_inputs as li
    import paper_1611_06365_gb300 as lu

    n = args.mixed_n
    hbm_peak = _measured_peaks().get("hbm_gbs", 6793.0)
    bf16_peak = _measured_peaks().get("bf16_tflops_sustained", 1722.0)
    t0 = time.perf_counter()
    Q_u, Vt = li.kappa_factors_torch(n, MIXED_FAMILY + (0 if n == 16384 else 1), n, dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    plan_bo = None
    cases = []
    tc_roof = None
    kappas = [float(k) for k in args.c3_kappas.split(",")] if args.c3_kappas else MIXED_KAPPAS
    nrhs_list = [int(q) for q in args.c3_nrhs.split(",")] if args.c3_nrhs else MIXED_NRHS
    for kappa in kappas:
        A = li.kappa_from_factors_torch(Q_u, Vt, kappa)
        anorm = A.abs().sum(0).max()
        fp64 = None
        for nrhs in sorted(nrhs_list):
            Xt = torch.from_numpy(li.uniform(n, nrhs, MIXED_FAMILY + 500 + nrhs)).to(dev)
            Xt[:, 0] = 1.0
            Xt = Xt.t().contiguous()                       # (nrhs, n): row q = right-hand side q
            B = (A.t() @ Xt.t()).t().contiguous()
            X = torch.zeros_like(B)
            lu.lu_solve_mixed(A, B, X)                     # warm-up
            torch.cuda.synchronize()
            reps = []
            for _ in range(2):
                w0 = time.perf_counter()
                rep = lu.lu_solve_mixed(A, B, X)
                torch.cuda.synchronize()
                reps.append((time.perf_counter() - w0, rep))
            wall, rep = min(reps, key=lambda r: r[0])
            R = B - (A.t() @ X.t()).t()
            eta = float((R.abs().amax(1) / (anorm * X.abs().amax(1) + B.abs().amax(1))).max())
            fwd = float((X - Xt).abs().max() / Xt.abs().max())
            if plan_bo is None:
                plan_bo = lu.lu_plan_info(lu.LU_F32, n, update=lu.LU_UPDATE_BF16X3)[1]["nb"]
            # attainable bound of the factorization: the split-BF16 products (three per pair) at
            # the sustained BF16 rate, or the FP32 trailing matrix streamed once per panel
            bound_ms = max(3 * flops_lu(n) / (bf16_peak * 1e12), (8.0 / 3.0) * n ** 3 / plan_bo / (hbm_peak * 1e9)) * 1e3
            entry = {"kappa": kappa, "nrhs": nrhs, "rung": rep.rung, "f32_refactor": rep.f32_refactor,
                     "cost_stop": rep.cost_stop, "t_fallback_ms": rep.t_fallback_ms, "iterations": rep.iterations,
                     "gmres_iters": rep.gmres_iters, "fell_back": rep.fell_back, "eta": eta,
                     "forward_error": fwd, "forward_error_est": getattr(rep, "forward_error_est", None),
                     "mixed_ms": rep.t_total_ms, "mixed_wall_ms": wall * 1e3, "factor_ms": rep.t_factor_ms,
                     "refine_ms": rep.t_refine_ms, "factor_bound_ms": bound_ms,
                     "factor_frac_of_bound": bound_ms / rep.t_factor_ms if rep.t_factor_ms > 0 else None}
            if fp64 is None:
                # the plain FP64 path to the same target: FP64 factorization with the DFMA
                # update, FP64 refinement; and the same with the emulated FP64 update
                fp64 = {}
                for key, native in (("fp64", 1), ("fp64emu", 0)):
                    X64 = torch.zeros_like(B)
                    rep64 = lu.lu_solve_mixed(A, B, X64, fp64_factor=1, fallback_native=native)
                    torch.cuda.synchronize()
                    R64 = B - (A.t() @ X64.t()).t()
                    eta64 = float((R64.abs().amax(1) / (anorm * X64.abs().amax(1) + B.abs().amax(1))).max())
                    fp64.update({f"{key}_ms": rep64.t_total_ms, f"{key}_iterations": rep64.iterations,
                                 f"{key}_eta": eta64})
            entry.update(fp64)
            entry["speedup_vs_fp64"] = fp64["fp64_ms"] / rep.t_total_ms if rep.t_total_ms > 0 else None
            entry["speedup_vs_fp64emu"] = fp64["fp64emu_ms"] / rep.t_total_ms if rep.t_total_ms > 0 else None
            cases.append(entry)
            if tc_roof is None:
                # the tensor-core update inside one more run, against the HBM roofline (C in FP32
                # read and written once per launch, staged operands read once)
                lu.lu_update_timing(True)
                lu.lu_solve_mixed(A, B, X)
                torch.cuda.synchronize()
                lu.lu_update_timing(False)
                u_n, u_ms, u_flops, u_bytes = lu.lu_update_timing_read()
                if u_ms > 0:
                    gbs = u_bytes / (u_ms / 1e3) / 1e9
                    tc_roof = {"bound": "hbm", "kernel": "gemm_update_tc<3>", "launches": u_n, "total_ms": u_ms,
                               "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                               "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json)"}
            del B, X, Xt, R
        del A
    del Q_u, Vt
    torch.cuda.empty_cache()
    head = next((c for c in cases if c["kappa"] == 1e5 and c["nrhs"] == 1), cases[0])
    return {"n": n, "reflectors_per_side": n, "target_eta": 1e-14, "generation_s": gen_s, "plan_nb": plan_bo,
            "cases": cases, "update_roofline": tc_roof,
            "mixed_ms": head["mixed_ms"], "fp64_ms": head["fp64_ms"], "speedup_vs_fp64": head["speedup_vs_fp64"]}


def fp8_large(args, dev):
    """Mixed solves with the FP8 e4m3 update at order --mixed-n (65536: FP64 A 32 GiB, FP32
    factors 16 GiB), nrhs = 16, A = U diag(s) V^T with 256 Householder reflectors per side;
    one JSON line per kappa with the ladder's report, the backward error recomputed here and
    the forward error against X_true (column 0 = ones, the others uniform [-1, 1))."""
    import torch

    import lu_inputs as li
    import paper_1611_06365_gb300 as lu

    n, nrhs = args.mixed_n, 16
    for ci, kappa in enumerate(float(k) for k in args.kappas.split(",")):
        seed = 20161106 + 1000 * 5 + ci
        t0 = time.perf_counter()
        A = li.kappa_matrix_torch(n, kappa, seed, MIXED_REFLECTORS, dev)
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        Xt = torch.from_numpy(li.uniform(n, nrhs, seed + 1)).to(dev)
        Xt[:, 0] = 1.0
        Xt = Xt.t().contiguous()                       # (nrhs, n): row q = right-hand side q
        B = (A.t() @ Xt.t()).t().contiguous()          # B = A X_true
        X = torch.zeros_like(B)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rep = lu.lu_solve_mixed(A, B, X, update=lu.LU_UPDATE_FP8)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t1
        R = B - (A.t() @ X.t()).t()
        eta = float((R.abs().amax(1) / (A.abs().sum(0).max() * X.abs().amax(1) + B.abs().amax(1))).max())
        fwd = float((X - Xt).abs().max() / Xt.abs().max())
        print(json.dumps({"case": "fp8_large", "n": n, "nrhs": nrhs, "kappa": kappa, "seed": seed,
                          "reflectors_per_side": MIXED_REFLECTORS, "gen_s": gen_s, "wall_s": wall, "eta": eta,
                          "forward_error": fwd, "report": rep.as_dict()}), flush=True)
        del A, B, X, Xt, R
        torch.cuda.empty_cache()


def cholesky_measure(n, dev, reps):
    """A = L L^T of an SPD matrix of order n ((B + B^T) / 2 + n I, B uniform [-1, 1)), with the
    DFMA and the emulated FP64 updates (and the emulated one without look-ahead): n^3 / 3 flop,
    CUDA events around each call, the best of reps - 1 after a warm-up, and a randomized residual
    probe of each factor."""
    import numpy as np
    import torch

    import lu_inputs as li
    import paper_1611_06365_gb300 as lu

    B = li.uniform_colmajor_torch(n, n, 20161106 + 9100, dev, torch.float64)
    A0 = (B + B.t()) / 2
    del B
    A0.diagonal().add_(float(n))
    A = torch.empty_like(A0)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    out = {"n": n, "matrix": "(B + B^T)/2 + n I, B uniform [-1, 1)"}
    for name, upd, la in (("dfma", lu.LU_UPDATE_NATIVE, 0), ("f64emu", lu.LU_UPDATE_F64EMU, 0),
                          ("f64emu_no_lookahead", lu.LU_UPDATE_F64EMU, -1)):
        best = None
        for rep in range(reps):
            A.copy_(A0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            lu.lu_cholesky(A, info, n, update=upd, lookahead=la)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if rep > 0 or reps == 1:
                best = ms if best is None else min(best, ms)
        L = torch.tril(A.t())
        w = torch.from_numpy(np.random.default_rng(5).standard_normal(n)).to(dev)
        r = A0.t() @ w - L @ (L.t() @ w)
        out[name] = {"ms": best, "gflops": n ** 3 / 3.0 / (best / 1e3) / 1e9, "info": int(info.item()),
                     "residual_probe": float(r.norm() / (A0.norm() * w.norm()))}
        del L, r
    del A, A0
    torch.cuda.empty_cache()
    return out


def measure_peaks(dev):
    """ALU peaks on this GPU: DFMA, DMMA and FFMA throughput probes (lu_peak_probe), each
    a launch of about a second after a short warm-up, with the SM clocks sampled
    during the probes; FP8 e4m3 and BF16 library GEMMs (torch) as context points."""
    import torch

    import paper_1611_06365_gb300 as lu

    out = {"gpu": torch.cuda.get_device_name(dev), "how": "lu_peak_probe: 4 CTAs x 256 threads per SM, "
           "DFMA: the compute loop of the tiled update (4 x 4 outputs per thread, operands from shared memory); "
           "FFMA: 8 register chains per thread; DMMA: 4 chains per warp; "
           "CUDA events around one launch"}
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    time.sleep(0.3)
    for name, kind, iters in (("dfma", lu.PROBE_DFMA, 1 << 15), ("dmma", lu.PROBE_DMMA, 1 << 19),
                              ("ffma", lu.PROBE_FFMA, 1 << 23)):
        lu.lu_peak_probe(kind, iters // 64)
        tf, ms = lu.lu_peak_probe(kind, iters)
        out[name] = {"tflops": tf, "ms": ms, "iters": iters}
    out["clocks"] = clocks.stop()
    lib_pts = {}
    try:
        m = 8192
        a = torch.randn(m, m, device=dev).to(torch.float8_e4m3fn)
        b = torch.randn(m, m, device=dev).to(torch.float8_e4m3fn).t()
        one = torch.ones((), device=dev)
        for _ in range(3):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        e1.record()
        torch.cuda.synchronize()
        lib_pts["fp8_e4m3_scaled_mm_8192"] = 2.0 * m ** 3 * 10 / (e0.elapsed_time(e1) / 1e3) / 1e12
    except Exception as exc:   # a library context point only
        lib_pts["fp8_e4m3_scaled_mm_8192"] = f"unavailable: {type(exc).__name__}"
    out["library_tflops"] = lib_pts
    return out


def early_term_measure(dev):
    """Early termination (section 4.2) against the same plan without it: lu_factor time
    (CUDA events on the caller's stream, so the host's wait for each panel's width is
    inside; best of three after a warm-up), panels, and how many stopped early.  One row
    per workload."""
    import torch

    import lu_inputs as li
    import paper_1611_06365_gb300 as lu

    cases = (("fp64_dfma", 4096, torch.float64, lu.LU_UPDATE_NATIVE),
             ("fp64_emulated", 8192, torch.float64, lu.LU_UPDATE_F64EMU),
             ("fp32_split_bf16", 16384, torch.float32, lu.LU_UPDATE_BF16X3))
    rows = []
    for name, n, tdt, update in cases:
        A0 = li.uniform_colmajor_torch(n, n, 5, dev, tdt)
        A = torch.empty_like(A0)
        ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
        info = torch.zeros(1, dtype=torch.int32, device=dev)
        row = {"case": "early_term", "workload": name, "n": n, "nb": 64, "nb_inner": 16}
        for et in (0, 1):
            times = []
            for rep in range(4):
                A.copy_(A0)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                lu.lu_factor(A, ipiv, info, nb=64, nb_inner=16, update=update, early_term=et)
                e1.record()
                torch.cuda.synchronize()
                if rep > 0:
                    times.append(e0.elapsed_time(e1))
            w = lu.lu_last_panel_widths()
            key = "et_on" if et else "et_off"
            ms = min(times)
            row[key] = {"ms": ms, "gflops": flops_lu(n) / (ms / 1e3) / 1e9, "panels": len(w),
                        "stopped_early": sum(1 for i, x in enumerate(w[:-1]) if x < 64),
                        "mean_width": sum(w) / len(w), "info": int(info.item())}
        rows.append(row)
        del A0, A
    torch.cuda.empty_cache()
    return rows


def run_case(args):
    """Single-kernel cases for profiling (one launch of the kernel of interest)."""
    import torch

    import lu_inputs as li
    import paper_1611_06365_gb300 as lu

    dev = torch.device("cuda", 0)
    if args.case != "torch_context":   # the library-context case runs torch only
        lu.build()
    if args.case == "tc_update":
        # split-BF16 trailing update, C 8192 x 8192 FP32 (256 MiB, larger than L2), K = 256
        m = n = 8192
        k = 256
        A = li.uniform_colmajor_torch(m, k, 1, dev, torch.float32)
        B = li.uniform_colmajor_torch(k, n, 2, dev, torch.float32)
        C = li.uniform_colmajor_torch(m, n, 3, dev, torch.float32)
        lu.lu_trailing_update(lu.LU_UPDATE_BF16X3, A, B, C, m, n, k)
    elif args.case == "fp64_factor":
        # FP64 factorization, n = 8192 (512 MiB) unless --n is given, by default with the plan
        # the autotuner picks for the large orders on GB300 (b_o = 64, an 8-CTA panel team)
        n = 8192 if args.n == N_MAIN else args.n
        A = li.uniform_colmajor_torch(n, n, 5, dev, torch.float64)
        ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
        info = torch.zeros(1, dtype=torch.int32, device=dev)
        lu.lu_factor(A, ipiv, info, nb=args.nb or 64, panel_ctas=args.panel_ctas or 8,
                     update=lu.LU_UPDATE_F64EMU if args.emu else lu.LU_UPDATE_NATIVE)
    elif args.case == "mixed_factor":
        # FP32 factorization with the split-BF16 update, n = 8192
        n = 8192
        A = li.uniform_colmajor_torch(n, n, 5, dev, torch.float32)
        ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
        info = torch.zeros(1, dtype=torch.int32, device=dev)
        lu.lu_factor(A, ipiv, info, update=lu.LU_UPDATE_BF16X3)
    elif args.case == "solve_f32":
        # FP32 factors of order 16384 (split-BF16 update), then one solve with one right-hand
        # side: the refinement step's triangular solves
        n = 16384
        A = li.uniform_colmajor_torch(n, n, 5, dev, torch.float32)
        ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
        info = torch.zeros(1, dtype=torch.int32, device=dev)
        lu.lu_factor(A, ipiv, info, update=lu.LU_UPDATE_BF16X3)
        b = torch.ones(1, n, dtype=torch.float32, device=dev)
        lu.lu_solve(A, ipiv, b)
    elif args.case == "torch_context":
        # library context (not a target): torch.linalg.lu_factor / solve on the same inputs
        for n, tdt in ((512, torch.float64), (16384, torch.float64), (16384, torch.float32)):
            A = li.uniform_colmajor_torch(n, n, 20161106 + 1000 * 2, dev, torch.float64).t().contiguous().to(tdt)
            b = A @ torch.ones(n, 1, dtype=tdt, device=dev)
            for name, fn in (("lu_factor", lambda: torch.linalg.lu_factor(A)),
                             ("solve", lambda: torch.linalg.solve(A, b))):
                fn()
                torch.cuda.synchronize()
                reps = 5 if n <= 4096 else 2
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    fn()
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                print(json.dumps({"case": "torch_context", "routine": f"torch.linalg.{name}", "n": n,
                                  "dtype": str(tdt).replace("torch.", ""), "ms": ms,
                                  "gflops": flops_lu(n) / (ms / 1e3) / 1e9}), flush=True)
    elif args.case == "fp8_large":
        fp8_large(args, dev)
        return
    elif args.case == "peaks":
        print(json.dumps(measure_peaks(dev)), flush=True)
        return
    elif args.case == "early_term":
        for row in early_term_measure(dev):
            print(json.dumps(row), flush=True)
        return
    elif args.case == "cholesky":
        print(json.dumps(dict({"case": "cholesky"}, **cholesky_measure(args.n, dev, 3))), flush=True)
        return
    elif args.case == "emu_update":
        # the emulated FP64 update alone: C 8192 x 8192 FP64 (512 MiB, larger than L2), K = 64
        m = n = 8192
        A = li.uniform_colmajor_torch(m, 64, 1, dev, torch.float64)
        B = li.uniform_colmajor_torch(64, n, 2, dev, torch.float64)
        C = li.uniform_colmajor_torch(m, n, 3, dev, torch.float64)
        for _ in range(2):
            lu.lu_trailing_update_f64(lu.LU_UPDATE_F64EMU, A, B, C, m, n, 64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lu.lu_trailing_update_f64(lu.LU_UPDATE_F64EMU, A, B, C, m, n, 64)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(json.dumps({"case": "emu_update", "ms": ms, "fp64_equiv_tflops": 2.0 * m * n * 64 / (ms / 1e3) / 1e12,
                          "c_gbs": 16.0 * m * n / (ms / 1e3) / 1e9}), flush=True)
        return
    elif args.case == "probe_dfma":
        # one short DFMA probe launch (for a counter capture of the FP64 pipe)
        tf, ms = lu.lu_peak_probe(lu.PROBE_DFMA, 1 << 11)
        print(json.dumps({"case": "probe_dfma", "tflops": tf, "ms": ms}), flush=True)
        return
    elif args.case == "c3_grid":
        # the mixed-precision time-to-solution grid alone, at order --mixed-n
        print(json.dumps({"case": "c3_grid", "time_to_solution": time_to_solution(args, dev)}), flush=True)
        return
    elif args.case in ("batched_f64", "batched_f32"):
        # the batched workload (10 000 orders in [16, 256]): one factorization launch
        import numpy as np
        tdt = torch.float64 if args.case == "batched_f64" else torch.float32
        code = lu.LU_F64 if args.case == "batched_f64" else lu.LU_F32
        sizes = li.batch_sizes(BATCH_COUNT, 16, 256, seed=BATCH_SEED)
        offs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)])
        roffs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64))])
        buf = li.uniform_colmajor_torch(1, int(offs[-1]), BATCH_SEED, dev, tdt).view(-1)
        for t in range(1, BATCH_COUNT, 2):             # odd members diagonally dominant
            n_t = int(sizes[t])
            buf[int(offs[t]):int(offs[t + 1])].view(n_t, n_t).diagonal().add_(n_t)
        esz = buf.element_size()
        ns = torch.tensor(sizes, dtype=torch.int32, device=dev)
        ptrA = torch.tensor([buf.data_ptr() + int(o) * esz for o in offs[:-1]], dtype=torch.int64, device=dev)
        ipiv = torch.zeros(int(roffs[-1]), dtype=torch.int32, device=dev)
        ptrP = torch.tensor([ipiv.data_ptr() + int(o) * 4 for o in roffs[:-1]], dtype=torch.int64, device=dev)
        info = torch.zeros(BATCH_COUNT, dtype=torch.int32, device=dev)
        lu.lu_factor_batched(code, ns, ptrA, ns, ptrP, info, 256)
    else:
        raise SystemExit(f"unknown case {args.case}")
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "ok": True}))


def make_parser():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_MAIN)
    ap.add_argument("--mixed-n", dest="mixed_n", type=int, default=MIXED_N)
    ap.add_argument("--cpu-n", dest="cpu_n", type=int, default=8192)
    ap.add_argument("--ref-n", dest="ref_n", type=int, default=2048)
    ap.add_argument("--skip-mixed", dest="skip_mixed", action="store_true")
    ap.add_argument("--skip-emu", dest="skip_emu", action="store_true",
                    help="skip the factorization with the emulated FP64 update")
    ap.add_argument("--skip-cpu", dest="skip_cpu", action="store_true")
    ap.add_argument("--skip-batched", dest="skip_batched", action="store_true")
    ap.add_argument("--skip-chol", dest="skip_chol", action="store_true", help="leave out the Cholesky line")
    ap.add_argument("--skip-et", dest="skip_et", action="store_true",
                    help="leave out the early-termination comparison")
    ap.add_argument("--skip-small", dest="skip_small", action="store_true",
                    help="skip the n = 512 latency measurement")
    ap.add_argument("--no-autotune", dest="no_autotune", action="store_true",
                    help="run the built-in plans instead of timing candidates first")
    ap.add_argument("--tune-budget-ms", dest="tune_budget_ms", type=float, default=15000.0,
                    help="device time the autotuner may spend per order")
    ap.add_argument("--tune-file", dest="tune_file", default=None,
                    help="tuning table: loaded (no tuning) if it exists, else written after tuning")
    ap.add_argument("--case", choices=["tc_update", "fp64_factor", "mixed_factor", "batched_f64", "batched_f32",
                                       "fp8_large", "solve_f32", "torch_context", "peaks", "c3_grid", "probe_dfma",
                                       "emu_update", "cholesky", "early_term"],
                    default=None,
                    help="run one profiling case instead of the benchmark (fp8_large: the order-65536 "
                         "FP8-update solves, one JSON line per kappa)")
    ap.add_argument("--kappas", default="1e3,1e6,1e12", help="condition numbers of the fp8_large case")
    ap.add_argument("--c3-kappas", dest="c3_kappas", default=None,
                    help="condition numbers of the time-to-solution grid (default 1e2,1e5,1e8)")
    ap.add_argument("--c3-nrhs", dest="c3_nrhs", default=None,
                    help="right-hand side counts of the time-to-solution grid (default 1,8)")
    ap.add_argument("--nb", type=int, default=0, help="outer panel width of the fp64_factor case (0: 64)")
    ap.add_argument("--emu", action="store_true", help="fp64_factor case with the emulated FP64 update")
    ap.add_argument("--panel-ctas", dest="panel_ctas", type=int, default=0,
                    help="panel team of the fp64_factor case (0: 8)")
    return ap


def main():
    args = make_parser().parse_args()
    if args.case:
        run_case(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
