"""Benchmark: LQR stage-solves/s at KKT rel-resid <= 1e-9 on B300.

Workload (the configuration the metric is quoted on): a batch of 1024
dual-regularized LQR instances, n_x = 12, n_u = 4, N = 256, delta log-uniform
in [1e-8, 1e-2]; 30% with a non-convex Q (two negative eigenvalues, pivots PD),
5% pivot-indefinite on purpose; synthetic, seeded (paper_2509_16370_b300.inputs).

One step = one rlqr_solve_batched call over the whole batch: FP32 Riccati
sweep with the FP64 pivot certificate, FP64 KKT residual, FP32 corrections with
FP64 accumulation until every instance reaches rel-resid <= 1e-9 (device-side
early exit), i.e. every row of the hot path.  Inputs (0.9 GB) exceed L2, so no
flush is needed between steps.  The plain FP64 GPU recursion on the same batch
is timed beside it, and the FP64 CPU oracle is the CPU baseline.  With N = 1
the line also carries the other configurations under "configs" (the small
single instance, the long horizon, the first 512 ragged instances and the
IPM on 8192 cart-double-pendulum trajectories), each with its own timing and
CPU baseline; --no-extras leaves them out.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --profile-instances K   # profiling case, no bench line
    python bench.py --residual-route 1      # fixed residual route (profiler runs)
    python bench.py --long-horizon          # the single long-horizon instance
    python bench.py --latency               # latency of the small single instance
    python bench.py --cross P               # cross-stage variables, p = P
    python bench.py --ipm K                 # the nonlinear IPM on K cart-double-pendulum instances
    python bench.py --warm-start K          # learned warm start trained on K IPM runs
    python bench.py --diag                  # general diagonal Delta_i
    python bench.py --ragged K              # the first K instances of the ragged batch
    python bench.py --ragged K --ragged-n 48   # only the n = 48 instances among them

--long-horizon measures the other workload of the path: one instance with
n_x = 32, n_u = 8, N = 65536 (delta = 1e-7, rho(A) = 0.99, Q and R with
condition number 1e4), rlqr_factor + rlqr_solve with the associative scan in
mixed precision (FP64 residual and refinement), beside the plain FP64
sequential recursion on the GPU.

Multi-GPU (torchrun): every rank solves its own copy of the batch (weak
scaling, no data-path collective); value = all ranks' stage-solves / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="batch of 1024 dual-regularized LQRs, n_x=12, n_u=4, N=256, "
                         "delta log-uniform [1e-8,1e-2], 30% non-convex Q, 5% pivot-indefinite",
                instances=1024, N=256, n_x=12, n_u=4, l2="inputs 0.9 GB > L2 (no flush needed)")
METRIC = "LQR stage-solves/s at KKT rel-resid <=1e-9 (mixed+batched; plain FP64 beside)"
TOL = 1e-9
FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12  # 2 DFMA/clk/SM at the max SM clock (fallback)


def _dist(backend: str = "nccl"):
    """(rank, world size, local rank) from the torchrun environment; joins the
    process group when there is more than one rank."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    if not dist.is_initialized():
        dist.init_process_group(backend)
    return rank, ws, local


def rank_max(value: float, world: int, device="cuda") -> float:
    """The largest of a per-rank value over all ranks (the slowest rank's time
    bounds the job); the value itself on one rank."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput of replicas: every rank processes units_per_rank
    in at most ms_max milliseconds."""
    return world * units_per_rank / (ms_max / 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu, self.rows, self.proc = gpu, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()  # the sampler runs before the timed region starts
            while not self.rows and time.time() - t0 < 3.0:
                time.sleep(0.02)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# DRAM bytes (read + write) per instance-stage of each kernel, from one ncu
# capture each (the sweep and the residual at 296 instances of this workload,
# the refinement pass at all 1024; the kernels as they are in this source;
# see profiles/), scaled by the stages a launch processes.
TRAFFIC_PER_STAGE = {"k_seq_fp32_solve": 7481.0, "k_residual_ff": 3920.0,
                     "k_solve_refine": 5000.0}
# Warp instructions per instance-stage of the FP32 warp sweep (backward +
# forward) from the same capture: the length of one instance's instruction
# stream, which one warp must issue in order.
SWEEP_INSTR_PER_STAGE = {"k_seq_fp32_solve": 1484.0}
SM_COUNT, SMSP_PER_SM = 148, 4


def kernel_models(n, m, stages):
    """Algorithmic work per launch of each kernel for the roofline.

    Bytes: the FP64 problem data every pass must read (Q, M, R, q, r, A, B, c:
    8 (2n^2 + 2nm + m^2 + 2n + m) B per stage) plus the FP64 solution it must
    write (x, u, y: 8 (2n + m) B) and one flag byte; 3649 B per stage at
    n = 12, m = 4.  FLOPs of the FP64 residual: 2 (3n^2 + 4nm + m^2) per stage
    (the products of Section "Residual Computation")."""
    data = 8 * (2 * n * n + 2 * n * m + m * m + 2 * n + m)
    out = 8 * (2 * n + m) + 1
    return {
        "k_seq_fp32_solve": ("hbm", (data + out) * stages, "GB/s"),
        "k_seq_fp64_solve": ("hbm", (data + out) * stages, "GB/s"),
        "k_solve_refine": ("hbm", (data + 2 * out) * stages, "GB/s"),
        "k_residual_fp64": ("alu", 2.0 * (3 * n * n + 4 * n * m + m * m) * stages, "TFLOP/s"),
        # float-float residual + FP64 control-pivot certificate: reads the
        # data, z and the stored FP32 G_i, writes res
        "k_residual_ff": ("hbm", (data + 2 * 8 * (2 * n + m) + 4 * m * m + 1) * stages, "GB/s"),
    }


def scan_flops_per_stage(n, m):
    """Algorithmic FLOPs per stage of the scan kernels (the build's counts of
    the paper's formulas): the chunk fold does one combination per stage
    (elimination of I + C P, 2n^3/3, two-sided solves 4n^3, five n x n
    products 10n^3); a finalize pass is one step of the recursion."""
    comb = 2.0 / 3.0 * n ** 3 + 4.0 * n ** 3 + 10.0 * n ** 3
    return {"k_scan_reduce": comb, "k_scan_finalize": seq_flops_per_stage(n, m)}


def seq_flops_per_stage(n, m):
    """Algorithmic FLOPs of one stage of the sequential recursion with
    symmetry exploited: 16/3 n^3 + 5 n^2 m + 3 n m^2 + 1/3 m^3."""
    return 16.0 / 3.0 * n ** 3 + 5.0 * n * n * m + 3.0 * n * m * m + m ** 3 / 3.0


def chain_bound(name, launch_ms, N, count, sm_mhz):
    """The bound of a one-warp-per-instance sweep below HBM: each instance is
    one warp's in-order instruction stream, and a scheduler issues at most one
    instruction per cycle, so with the batch's warps spread over the 148 x 4
    schedulers the busiest scheduler holds ceil(count / 592) of them and a
    stage cannot take fewer than that many times the stream's instructions
    per stage in cycles.  frac = that floor / the measured cycles per stage."""
    ipst = SWEEP_INSTR_PER_STAGE.get(name)
    if not ipst or not sm_mhz:
        return None
    per_sched = -(-count // (SM_COUNT * SMSP_PER_SM))
    cycles = launch_ms * 1e-3 * sm_mhz * 1e6 / N
    floor = per_sched * ipst
    return {"bound": "instruction issue of the per-instance chains",
            "instr_per_stage": ipst, "warps_on_busiest_scheduler": per_sched,
            "floor_cycles_per_stage": floor, "cycles_per_stage": round(cycles, 1),
            "frac": round(floor / cycles, 4),
            "issue_rate_frac_of_gpu": round(ipst * N * count / (launch_ms * 1e-3) /
                                            (SM_COUNT * SMSP_PER_SM * sm_mhz * 1e6), 4)}


def roofline(report, steps, n, m, stages, peaks, fp64_tflops=None, chain=None):
    k = [(ms, name, cnt) for name, (cnt, ms) in report.items() if name != "k_plan"]
    if not k:
        return None
    ms, name, cnt = max(k)
    bound, work, unit = kernel_models(n, m, stages).get(name, ("hbm", 0.0, "GB/s"))
    per_launch_s = ms / cnt / 1e3
    if bound == "hbm":
        achieved = work / per_launch_s / 1e9
        peak = float(peaks.get("hbm_gbs", 6400.0))
        peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    else:
        achieved = work / per_launch_s / 1e12
        peak = fp64_tflops or FP64_PEAK_TFLOPS
        peak_src = ("measured FP64 FMA rate (rlqr_measure_pipes)" if fp64_tflops
                    else "derived (148 SM x 2 FP64 FMA/clk x 2032 MHz)")
    total = sum(v[1] for v in report.values())
    traffic = TRAFFIC_PER_STAGE.get(name)
    out = {"kernel": name, "bound": bound, "achieved": round(achieved, 3), "peak": peak,
           "peak_source": peak_src, "unit": unit, "frac": round(achieved / peak, 4),
           "traffic": None if traffic is None else traffic * stages,
           "algorithmic_bytes": work if bound == "hbm" else None,
           "launch_ms": round(ms / cnt, 4), "share": round(ms / total, 3)}
    if chain:
        N, count, sm_mhz = chain
        cb = chain_bound(name, ms / cnt, N, count, sm_mhz)
        if cb:
            # the kernel is bound by its chains, not by HBM: the HBM fraction
            # stays the reported one, and it is far from one half
            out["chain"] = cb
            out["hbm_frac_at_least_half"] = bool(achieved / peak >= 0.5) if bound == "hbm" else None
    return out


def fp64_sweep_roofline(report, n, m, stages, pipes):
    """The plain FP64 sweep against the measured FP64 FMA rate (the pipe that
    bounds it on B300): algorithmic FLOPs of the recursion / launch time."""
    name = "k_seq_fp64_solve"
    if name not in report:
        return None
    cnt, ms = report[name]
    achieved = seq_flops_per_stage(n, m) * stages / (ms / cnt / 1e3) / 1e12
    peak = pipes["fp64_tflops"]
    return {"kernel": name, "bound": "fp64", "achieved": round(achieved, 4),
            "peak": round(peak, 4), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
            "peak_source": "measured FP64 FMA rate (rlqr_measure_pipes)",
            "flops_per_stage": round(seq_flops_per_stage(n, m), 1)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_baseline(bh, min_seconds=10.0):
    """The FP64 oracle's sequential recursion (OpenMP over instances) on the
    same batch, repeated until ~min_seconds of CPU work."""
    import oracle
    oracle.riccati_batch(bh)  # warm (builds the oracle if needed)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.riccati_batch(bh)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds or reps >= 200:
            break
    stages = bh.count * bh.N * reps
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": stages / dt, "unit": "stage-solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} x full batch ({bh.count} instances x N={bh.N}), {dt:.1f} s",
            "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "build": "gcc " + " ".join(oracle.CFLAGS)}


def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo), or "unknown"."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args):
    # The oracle is a host program: under torchrun only rank 0 runs it.
    if int(os.environ.get("RANK", "0")) != 0:
        return
    from paper_2509_16370_b300 import inputs
    import oracle
    bh = inputs.workload2()
    for _ in range(args.warmup):
        oracle.riccati_batch(bh)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.riccati_batch(bh)
    dt = time.perf_counter() - t0
    value = bh.count * bh.N * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"metric": METRIC, "value": value, "unit": "stage-solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": WORKLOAD, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "stage-solves/s", "cores": cores,
                             "kind": "oracle", "sample": f"full batch per step, {args.steps} steps"},
            "e2e": {"value": value, "unit": "stage-solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """The mixed solve alone on the first K instances of the workload: warm-up
    calls, then one call (the launch an ncu capture selects with -s/-c)."""
    import torch
    from paper_2509_16370_b300 import inputs, rlqr
    bh = inputs.workload2(count=args.profile_instances)
    db = rlqr.DeviceBatch.from_uniform(bh)
    opts = rlqr.make_opts(rlqr.RLQR_MIXED, tol=TOL, max_refine=3)
    ws = rlqr.alloc_workspace(rlqr.rlqr_batched_workspace_bytes(db, opts))
    B = bh.count
    st = torch.zeros(B, dtype=torch.int32, device="cuda")
    rel = torch.zeros(B, dtype=torch.float64, device="cuda")
    it = torch.zeros(B, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup + 1):
        rlqr.rlqr_solve_batched(db, opts, ws, st, rel, it)
    torch.cuda.synchronize()
    print(f"profile case: {B} instances, max rel {rel.max().item():.3e}, "
          f"iters {it.max().item()}", flush=True)


def run_latency(args):
    print(json.dumps(measure_latency(args)), flush=True)


def measure_latency(args):
    """The small single instance (n=4, m=2, N=64): the latency of
    rlqr_factor + rlqr_solve per call, launched one call after another and
    replayed from a CUDA graph of the same calls, FP64 and mixed (with
    refinement).  The configuration is bound by launch latency, not by a pipe
    or HBM, so no roofline fraction is given.  CPU baseline: the oracle's
    recursion on the same instance, one core."""
    import torch
    import oracle
    from paper_2509_16370_b300 import inputs, rlqr
    p = inputs.workload1()
    dp = rlqr.DeviceProblem.from_host(p)
    N, n, m = p.N, p.n, p.m
    out = {}
    for name, prec, algo in (("fp64_seq", rlqr.RLQR_FP64, rlqr.RLQR_ALGO_SEQ),
                             ("mixed_seq", rlqr.RLQR_MIXED, rlqr.RLQR_ALGO_SEQ),
                             ("fp64_scan", rlqr.RLQR_FP64, rlqr.RLQR_ALGO_SCAN),
                             ("mixed_scan", rlqr.RLQR_MIXED, rlqr.RLQR_ALGO_SCAN)):
        opts = rlqr.make_opts(prec, algo=algo, tol=TOL, max_refine=3)
        ws = rlqr.alloc_workspace(rlqr.rlqr_workspace_bytes(N, n, m, opts))
        flags = torch.zeros(N + 1, dtype=torch.uint8, device="cuda")
        x = torch.zeros(N + 1, n, dtype=torch.float64, device="cuda")
        u = torch.zeros(N, m, dtype=torch.float64, device="cuda")
        y = torch.zeros(N + 1, n, dtype=torch.float64, device="cuda")
        rel = torch.zeros(1, dtype=torch.float64, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())

        def call():
            rlqr.rlqr_factor(dp, opts, ws, flags)
            rlqr.rlqr_solve(dp, opts, ws, x, u, y, rel)

        with torch.cuda.stream(side):
            for _ in range(args.warmup):
                call()
        torch.cuda.synchronize()
        reps = max(args.steps, 20)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(side):
            e0.record(side)
            for _ in range(reps):
                call()
            e1.record(side)
        torch.cuda.synchronize()
        eager_us = e0.elapsed_time(e1) / reps * 1e3
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            call()
        g.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        graph_us = e0.elapsed_time(e1) / reps * 1e3
        out[name] = {"eager_us_per_call": round(eager_us, 2), "graph_us_per_call": round(graph_us, 2),
                     "rel_resid": float(rel.item())}
    best = min(out, key=lambda k: out[k]["graph_us_per_call"])
    oracle.riccati(p)
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < 1.0:
        oracle.riccati(p)
        reps += 1
    cpu_s = (time.perf_counter() - t0) / reps
    mixed_us = min(out["mixed_seq"]["graph_us_per_call"], out["mixed_scan"]["graph_us_per_call"])
    line = {"metric": "latency of one factor + solve (n=4, m=2, N=64)",
            "value": out[best]["graph_us_per_call"], "unit": "us", "higher_is_better": False,
            "n_gpus": 1, "steps": max(args.steps, 20), "warmup": args.warmup, "data": "synthetic",
            "config": {"workload": "single instance n_x=4, n_u=2, N=64, delta=1e-6", "best": best},
            "stage_solves_per_s": {"mixed": N / (mixed_us * 1e-6),
                                   "fp64": N / (min(out["fp64_seq"]["graph_us_per_call"],
                                                    out["fp64_scan"]["graph_us_per_call"]) * 1e-6)},
            "roofline": None,
            "roofline_note": "launch-latency bound: 37 KB of data, a chain of 64 stages",
            "cpu_baseline": {"value": N / cpu_s, "unit": "stage-solves/s", "cores": 1,
                             "kind": "oracle", "sample": f"{reps} x the instance, 1 s",
                             "us_per_call": round(cpu_s * 1e6, 2)},
            **out}
    return line


def run_cross(args):
    """One JSON line for cross-stage variables (Section "Cross-Stage
    Variables"): one instance of the batch workload (n=12, m=4, N=256),
    factored once; the time of rlqr_solve_cross for p shared variables (p + 1
    solves with the factor, the Schur complement and the combination) beside
    one plain rlqr_solve, mixed precision with refinement."""
    import torch
    from paper_2509_16370_b300 import inputs, rlqr
    prob = inputs.random_instance(900, 256, 12, 4, 1e-4)
    dp = rlqr.DeviceProblem.from_host(prob)
    N, n, m, p = prob.N, prob.n, prob.m, args.cross
    opts = rlqr.make_opts(rlqr.RLQR_MIXED, algo=rlqr.RLQR_ALGO_SEQ, tol=TOL, max_refine=3)
    ws = rlqr.alloc_workspace(rlqr.rlqr_workspace_bytes(N, n, m, opts))
    flags = torch.zeros(N + 1, dtype=torch.uint8, device="cuda")
    rlqr.rlqr_factor(dp, opts, ws, flags)
    g = torch.Generator(device="cpu").manual_seed(900)
    L = 2 * (N + 1) * n + N * m
    J = torch.randn(p, L, generator=g, dtype=torch.float64).cuda()
    Hs = torch.randn(p, p, generator=g, dtype=torch.float64)
    H = (Hs + Hs.T + 2 * p * torch.eye(p, dtype=torch.float64)).cuda()
    rt = torch.randn(p, generator=g, dtype=torch.float64).cuda()
    sc = rlqr.alloc_workspace(rlqr.rlqr_cross_scratch_bytes(N, n, m, p, opts))
    x = torch.zeros(N + 1, n, dtype=torch.float64, device="cuda")
    u = torch.zeros(N, m, dtype=torch.float64, device="cuda")
    y = torch.zeros(N + 1, n, dtype=torch.float64, device="cuda")
    dth = torch.zeros(p, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")

    def timeit(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    ms_cross = timeit(lambda: rlqr.rlqr_solve_cross(dp, opts, ws, J, H, rt, sc, x, u, y, dth, st))
    ms_solve = timeit(lambda: rlqr.rlqr_solve(dp, opts, ws, x, u, y))
    line = {"metric": "cross-stage solve time (p shared variables, one factor)",
            "value": ms_cross, "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
            "config": {"workload": "single instance n_x=12, n_u=4, N=256, delta=1e-4",
                       "p": p, "precision": "mixed"},
            "plain_solve_ms": ms_solve, "ratio_to_plain_solve": ms_cross / ms_solve,
            "status": int(st.item())}
    if not args.no_cpu_baseline:
        import oracle
        Jh = J.cpu().numpy()
        nX, nU = (N + 1) * n, N * m
        Jq = Jh[:, :nX].reshape(p, N + 1, n)
        Jr = Jh[:, nX:nX + nU].reshape(p, N, m)
        Jc = Jh[:, nX + nU:].reshape(p, N + 1, n)
        t0 = time.time()
        oracle.cross_stage_solve(prob, Jq, Jr, Jc, H.cpu().numpy(), rt.cpu().numpy())
        line["cpu_baseline"] = {"value": (time.time() - t0) * 1e3, "unit": "ms", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": "one dense bordered solve (numpy LAPACK)"}
    print(json.dumps(line), flush=True)


def run_ipm(args):
    print(json.dumps(measure_ipm(args)), flush=True)


def measure_ipm(args):
    """One JSON line for the regularized interior-point method (Section "The
    Regularized Interior Point Method", Section "Applying the regularized IPM
    to optimal control") on the first K cart-double-pendulum instances
    (N = 128, n_x = 6, n_u = 1, RK4 dt = 0.02; angles uniform in [-pi, pi]).
    One step = one whole solve from the cold start (rollout of u = 0) to
    convergence or the iteration limit, with the FP32 Hessian and the
    mixed-precision LQR solves; warm-up = one solve of 64 instances.  Reports
    instance-iterations/s, the LQR stage-solves/s inside the IPM, the share
    converged and their mean iteration count, beside the oracle's IPM on the
    host cores (a few instances)."""
    import torch
    from paper_2509_16370_b300 import inputs, ipm
    count = args.ipm
    x0, xg = inputs.workload5(count)
    model = ipm.make_model()
    kw = {"max_iter": args.ipm_max_iter} if args.ipm_max_iter else {}
    kw["hessian"] = {"fp32": ipm.RLQR_IPM_HESS_EXACT_FP32, "fp64": ipm.RLQR_IPM_HESS_EXACT_FP64,
                     "gn": ipm.RLQR_IPM_HESS_GAUSS_NEWTON}[args.ipm_hessian]
    opts = ipm.make_ipm_opts(**kw)
    st = ipm.IpmState(count, model.N)
    ws = ipm.alloc_ipm_workspace(count, model, opts)
    dx0, dxg = torch.from_numpy(x0).cuda(), torch.from_numpy(xg).cuda()
    wst = ipm.IpmState(64, model.N)
    wws = ipm.alloc_ipm_workspace(64, model, opts)
    ipm.rlqr_ipm_init(model, opts, dx0[:64].contiguous(), wst)
    ipm.rlqr_ipm_solve(model, opts, dx0[:64].contiguous(), dxg[:64].contiguous(), wst, wws)
    torch.cuda.synchronize()
    ms, n_it = [], 0
    with ClockSampler(0) as clocks:
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ipm.rlqr_ipm_init(model, opts, dx0, st)
            n_it = ipm.rlqr_ipm_solve(model, opts, dx0, dxg, st, ws)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    status = st.status.cpu().numpy()
    iters = st.iters.cpu().numpy()
    facts = st.factorizations.cpu().numpy()
    t = float(np.median(ms)) / 1e3
    conv = status == ipm.CONVERGED
    line = {"metric": "IPM instance-iterations/s (regularized IPM, cart-double-pendulum)",
            "value": float(iters.sum()) / t, "unit": "instance-iterations/s",
            "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": 1,
            "ms_per_step": t * 1e3, "dtype": {"fp32": "f64 (FP32 Hessian term, mixed LQR)",
                                                    "fp64": "f64 (FP64 Hessian term, mixed LQR)",
                                                    "gn": "f64 (Gauss-Newton Hessian, mixed LQR)"
                                                    }[args.ipm_hessian],
            "data": "synthetic",
            "config": {"workload": f"{count} cart-double-pendulum trajectories, N=128, n_x=6, "
                                   "n_u=1, RK4 dt=0.02, |u|<=20, |p|<=2, angles U[-pi,pi]",
                       "instances": count, "max_iter": opts.max_iter, "tol": opts.tol},
            "iterations_run": n_it, "ms_per_iteration": t * 1e3 / max(n_it, 1),
            "lqr_stage_solves_per_s": float(facts.sum()) * model.N / t,
            "factorizations_per_iteration": float(facts.sum() / max(iters.sum(), 1)),
            "converged_fraction": float(conv.mean()),
            "mean_iterations_converged": float(iters[conv].mean()) if conv.any() else None,
            "status_counts": {k: int((status == v).sum()) for k, v in
                              (("converged", 1), ("iteration_limit", 2), ("rho_limit", 3))},
            "roofline": None,
            "roofline_note": "the iteration's dominant kernels (k_ipm_step, k_ipm_lin) are bound "
                             "by the FP64 pipe (82-84 % busy in their ncu captures under "
                             "profiles/); no algorithmic flop count of the nonlinear model "
                             "is kept, so no live fraction is given",
            "clocks": clocks.summary()}
    if not args.no_cpu_baseline:
        import oracle.ipm as O
        md, op = O.Model(), O.Options()
        t0, done, it_sum = time.time(), 0, 0
        while time.time() - t0 < args.cpu_seconds and done < count:
            r = O.solve(md, op, x0[done], xg[done])
            it_sum += r.iters
            done += 1
        el = time.time() - t0
        line["cpu_baseline"] = {"value": it_sum / el, "unit": "instance-iterations/s",
                                "cores": 1, "kind": "oracle",
                                "sample": f"{done} whole solves (instances 0..{done - 1})"}
    return line


def wilson(k, n, z=1.96):
    """Wilson score interval of a binomial proportion k / n (95 %)."""
    if n == 0:
        return None
    p = k / n
    d = 1.0 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * np.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return [round(float(c - h), 4), round(float(c + h), 4)]


def run_ipm_study(args):
    """Why cold IPM solves stop short: one JSON line for the first K
    cart-double-pendulum instances (cold start, the default options, 300
    iterations).  Reports the converged share with its 95 % Wilson interval,
    the iteration quantiles of the converged instances, the final KKT error,
    dynamics defect (max |c| of the last Newton system, the linearization's
    own residual) and bound violation of the rest, whether the zero-force
    rollout of the initial point stays inside the bounds (then the problem
    has a feasible point and a stop is not infeasibility), and the share of
    the non-converged instances that converge when the same start is given
    1000 iterations, a doubled force bound, a doubled cart bound or a
    doubled horizon."""
    import torch
    from paper_2509_16370_b300 import inputs, ipm
    count = args.ipm_study
    x0, xg = inputs.workload5(count)
    base = dict(inputs.CDP_MODEL)

    def solve(idx, max_iter=300, **mk):
        model = ipm.make_model(**mk)
        opts = ipm.make_ipm_opts(max_iter=max_iter)
        st = ipm.IpmState(len(idx), model.N)
        ws = ipm.alloc_ipm_workspace(len(idx), model, opts)
        dx0 = torch.from_numpy(x0[idx]).cuda().contiguous()
        dxg = torch.from_numpy(xg[idx]).cuda().contiguous()
        ipm.rlqr_ipm_init(model, opts, dx0, st)
        X_init = st.X.clone()
        t0 = time.perf_counter()
        ipm.rlqr_ipm_solve(model, opts, dx0, dxg, st, ws)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        v = ipm.rlqr_ipm_lqr_view(model, opts, st, ws)
        return dict(model=model, st=st, X_init=X_init.cpu().numpy(),
                    status=st.status.cpu().numpy(), iters=st.iters.cpu().numpy(),
                    kkt=st.kkt.cpu().numpy(), defect=v["c"].abs().amax(dim=(1, 2)).cpu().numpy(),
                    X=st.X.cpu().numpy(), U=st.U.cpu().numpy(), seconds=el)

    idx = np.arange(count)
    r = solve(idx)
    conv = r["status"] == ipm.CONVERGED
    nc = np.flatnonzero(~conv)
    pmax, umax = base["p_max"], base["u_max"]
    bound_viol = np.maximum(np.maximum(np.abs(r["U"]).max(1) - umax,
                                       np.abs(r["X"][:, :, 0]).max(1) - pmax), 0.0)
    init_inside = np.abs(r["X_init"][:, :, 0]).max(1) <= pmax

    def q(v):
        v = np.asarray(v, dtype=float)
        if v.size == 0:
            return None
        return {k: float(np.quantile(v, p)) for k, p in
                (("min", 0.0), ("q10", 0.1), ("median", 0.5), ("q90", 0.9), ("max", 1.0))}

    relaxed = {}
    if nc.size:
        for name, kw in (("iterations_1000", dict(max_iter=1000)),
                         ("u_max_x2", dict(u_max=2 * umax)),
                         ("p_max_x2", dict(p_max=2 * pmax)),
                         ("horizon_x2", dict(N=2 * base["N"]))):
            mi = kw.pop("max_iter", 300)
            rr = solve(nc, max_iter=mi, **kw)
            k = int((rr["status"] == ipm.CONVERGED).sum())
            relaxed[name] = {"converged": k, "of": int(nc.size),
                             "fraction": round(k / nc.size, 4), "ci95": wilson(k, nc.size),
                             "mean_iterations_converged":
                                 float(rr["iters"][rr["status"] == ipm.CONVERGED].mean())
                                 if k else None}
    line = {"metric": "IPM cold-start convergence study (cart-double-pendulum)",
            "config": {"workload": f"the first {count} cart-double-pendulum instances, N=128, "
                                   "n_x=6, n_u=1, RK4 dt=0.02, |u|<=20, |p|<=2, angles U[-pi,pi]",
                       "max_iter": 300, "tol": 1e-6},
            "converged": int(conv.sum()), "instances": count,
            "converged_fraction": round(float(conv.mean()), 4),
            "converged_ci95": wilson(int(conv.sum()), count),
            "status_counts": {k: int((r["status"] == v).sum()) for k, v in
                              (("converged", ipm.CONVERGED), ("iteration_limit", ipm.ITERATION_LIMIT),
                               ("rho_limit", ipm.RHO_LIMIT))},
            "iterations_converged": q(r["iters"][conv]),
            "not_converged": {"final_kkt": q(r["kkt"][nc]), "dynamics_defect": q(r["defect"][nc]),
                              "bound_violation": q(bound_viol[nc])},
            "zero_force_rollout_inside_bounds": {"all": int(init_inside.sum()),
                                                 "not_converged": int(init_inside[nc].sum())},
            "relaxed_from_the_same_start": relaxed,
            "seconds_cold_solve": round(r["seconds"], 3)}
    print(json.dumps(line), flush=True)


def run_warm_start(args):
    """One JSON line for the learned warm start of the IPM: cold-start solves
    of the first K cart-double-pendulum instances give the training set (the
    converged ones: (x0, goal) -> (X, U)); the BF16 network of
    include/rlqr_mlp.h (3 layers, width 256) is trained on the GPU by its own
    kernels; then 8192 held-out instances (from index 1,000,000) are solved
    from the cold start and from the network's proposal.  Reports converged
    share and mean iterations, cold vs warm."""
    import torch
    from paper_2509_16370_b300 import inputs, ipm, mlp
    K, B = args.warm_start, 8192
    model, opts = ipm.make_model(), ipm.make_ipm_opts()
    N = model.N
    st = ipm.IpmState(B, N)
    ws = ipm.alloc_ipm_workspace(B, model, opts)
    t0 = time.time()
    feats, outs, solved = [], [], 0
    for s0 in range(0, K, B):
        x0, xg = inputs.workload5(B, s0)
        dx0, dxg = torch.from_numpy(x0).cuda(), torch.from_numpy(xg).cuda()
        ipm.rlqr_ipm_init(model, opts, dx0, st)
        ipm.rlqr_ipm_solve(model, opts, dx0, dxg, st, ws)
        ok = (st.status == ipm.CONVERGED).cpu().numpy()
        solved += int(ok.sum())
        feats.append(mlp.features(x0[ok], xg[ok]))
        outs.append(mlp.targets(st.X.cpu().numpy()[ok], st.U.cpu().numpy()[ok]))
    t_data = time.time() - t0
    F, T = np.concatenate(feats), np.concatenate(outs)
    norm = mlp.Normalizer(T)
    d = mlp.make_dims(mlp.N_IN, 256, T.shape[1], 256)
    net = mlp.WarmStartNet(d, mlp.init_params(d, 2025))
    Xd = torch.from_numpy(F).cuda()
    Td = torch.from_numpy(norm.encode(T)).cuda()
    torch.cuda.synchronize()
    # the launch-bound training step: eager launches against one CUDA graph
    # replayed per step (the same kernels; both timed on a 400-step copy)
    probe = {}
    for name, fn in (("eager", mlp.train), ("graph", mlp.train_graph)):
        pn = mlp.WarmStartNet(d, mlp.init_params(d, 2025))
        torch.cuda.synchronize()
        tp = time.time()
        fn(pn, Xd, Td, steps=400, batch=256, lr=1e-3, lr_final=5e-5, seed=7)
        torch.cuda.synchronize()
        probe[name] = 400 / (time.time() - tp)
        del pn
    t1 = time.time()
    losses = mlp.train_graph(net, Xd, Td, steps=args.ws_steps, batch=256, lr=1e-3,
                             lr_final=5e-5, seed=7)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    x0, xg = inputs.workload5(B, 1_000_000)
    dx0, dxg = torch.from_numpy(x0).cuda(), torch.from_numpy(xg).cuda()
    res, per = {}, {}
    for kind in ("cold", "warm"):
        t2 = time.time()
        if kind == "cold":
            ipm.rlqr_ipm_init(model, opts, dx0, st)
        else:
            X0, U0 = mlp.propose(net, norm, x0, xg, N)
            ipm.rlqr_ipm_init(model, opts, dx0, st, U0=U0, X0=X0)
        ipm.rlqr_ipm_solve(model, opts, dx0, dxg, st, ws)
        torch.cuda.synchronize()
        status, iters = st.status.cpu().numpy(), st.iters.cpu().numpy()
        conv = status == ipm.CONVERGED
        per[kind] = (conv, iters)
        res[kind] = {"converged_fraction": float(conv.mean()),
                     "mean_iterations_converged": float(iters[conv].mean()) if conv.any() else None,
                     "mean_iterations_all": float(iters.mean()),
                     "solve_s": time.time() - t2}
    both = per["cold"][0] & per["warm"][0]
    line = {"metric": "IPM mean iterations to convergence, cold vs learned warm start",
            "value": res["warm"]["mean_iterations_all"], "unit": "iterations (all instances, "
            "capped at max_iter)", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "cart-double-pendulum, N=128, angles U[-pi,pi]; training "
                                   f"runs {K}, held-out 8192",
                       "network": "3 layers, width 256, BF16 weights/activations, Adam",
                       "train_steps": args.ws_steps, "batch": 256},
            "cold": res["cold"], "warm": res["warm"],
            "paired": {"instances_converged_both": int(both.sum()),
                       "mean_iterations_cold": float(per["cold"][1][both].mean()) if both.any() else None,
                       "mean_iterations_warm": float(per["warm"][1][both].mean()) if both.any() else None,
                       "converged_warm_only": int((per["warm"][0] & ~per["cold"][0]).sum()),
                       "converged_cold_only": int((per["cold"][0] & ~per["warm"][0]).sum())},
            "training_solutions": int(F.shape[0]),
            "training_runs": K, "data_s": t_data, "train_s": t_train,
            "loss_first": losses[0], "loss_last": losses[-1]}
    if not args.no_cpu_baseline:
        import oracle.mlp as OM
        p = net.p.cpu().numpy().astype(np.float64)
        mm, vv = np.zeros_like(p), np.zeros_like(p)
        Tn = norm.encode(T).astype(np.float64)
        rng = np.random.default_rng(7)
        t0, k = time.time(), 0
        while time.time() - t0 < 10.0:
            idx = rng.choice(F.shape[0], 256, replace=False)
            _, g = OM.loss_and_grad(p, F[idx].astype(np.float64), Tn[idx], T.shape[1], 256)
            p, mm, vv = OM.adam(p, mm, vv, g, k + 1, 1e-3)
            k += 1
        el = time.time() - t0
        line["cpu_baseline"] = {"value": k / el, "unit": "training steps/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": f"{k} oracle training steps (batch 256, "
                                "FP64 numpy with BF16 rounding)"}
        line["gpu_training_steps_per_s"] = args.ws_steps / t_train
    line["training_steps_per_s"] = {"graph_replay": round(probe["graph"], 1),
                                    "eager_launches": round(probe["eager"], 1),
                                    "launches_per_step": 19}
    print(json.dumps(line), flush=True)


def run_diag(args):
    """One JSON line for the general diagonal Delta_i (rlqr_solve_diag: the
    congruence scaling, factor + solve of the scaled copy, the map back)
    beside rlqr_factor + rlqr_solve with scalar delta, on one instance of the
    batch workload's size (n=12, m=4, N=256), mixed precision."""
    import torch
    from paper_2509_16370_b300 import inputs, rlqr
    prob = inputs.random_instance(901, 256, 12, 4, 1e-4)
    N, n, m = prob.N, prob.n, prob.m
    dp = rlqr.DeviceProblem.from_host(prob)
    opts = rlqr.make_opts(rlqr.RLQR_MIXED, algo=rlqr.RLQR_ALGO_SEQ, tol=TOL, max_refine=3)
    d = torch.from_numpy(10.0 ** np.random.default_rng(901).uniform(-6, -2, (N + 1, n))).cuda()
    wsd = rlqr.alloc_workspace(rlqr.rlqr_diag_workspace_bytes(N, n, m, opts))
    ws = rlqr.alloc_workspace(rlqr.rlqr_workspace_bytes(N, n, m, opts))
    f = dict(dtype=torch.float64, device="cuda")
    x, u, y = torch.zeros(N + 1, n, **f), torch.zeros(N, m, **f), torch.zeros(N + 1, n, **f)
    flags = torch.zeros(N + 1, dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")

    def timeit(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    def plain():
        rlqr.rlqr_factor(dp, opts, ws, flags)
        rlqr.rlqr_solve(dp, opts, ws, x, u, y)

    ms_diag = timeit(lambda: rlqr.rlqr_solve_diag(dp, d, opts, wsd, x, u, y, flags, None, st))
    ms_plain = timeit(plain)
    line = {"metric": "factor + solve time with diagonal Delta_i (scaled copy) vs scalar delta",
            "value": ms_diag, "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
            "config": {"workload": "single instance n_x=12, n_u=4, N=256, Delta_i entries "
                                   "10^U(-6,-2)", "precision": "mixed"},
            "scalar_delta_ms": ms_plain, "ratio": ms_diag / ms_plain, "status": int(st.item())}
    if not args.no_cpu_baseline:
        import oracle
        dh = d.cpu().numpy()
        t0, k = time.time(), 0
        while time.time() - t0 < 2.0:
            oracle.riccati_diag(prob, dh)
            k += 1
        line["cpu_baseline"] = {"value": (time.time() - t0) * 1e3 / k, "unit": "ms", "cores": 1,
                                "kind": "oracle", "sample": f"{k} general-Delta recursions (numpy)"}
    print(json.dumps(line), flush=True)


def run_long_horizon(args):
    print(json.dumps(measure_long_horizon(args)), flush=True)


def measure_long_horizon(args, fp64_reps=1, fp64_warmup=1):
    """The long-horizon instance (stage-solves/s of factor + solve +
    refinement; SCAN mixed vs SEQ FP64 on the GPU).  CPU baseline: the
    oracle's recursion on the first 4096 stages (one core)."""
    import torch
    import oracle
    from paper_2509_16370_b300 import inputs, rlqr
    p = inputs.workload3(N=getattr(args, "lh_stages", 65536))
    dp = rlqr.DeviceProblem.from_host(p)
    N, n, m = p.N, p.n, p.m

    def make(prec, algo):
        opts = rlqr.make_opts(prec, algo=algo, tol=TOL, max_refine=3)
        ws = rlqr.alloc_workspace(rlqr.rlqr_workspace_bytes(N, n, m, opts))
        bufs = dict(flags=torch.zeros(N + 1, dtype=torch.uint8, device="cuda"),
                    x=torch.zeros(N + 1, n, dtype=torch.float64, device="cuda"),
                    u=torch.zeros(N, m, dtype=torch.float64, device="cuda"),
                    y=torch.zeros(N + 1, n, dtype=torch.float64, device="cuda"),
                    rel=torch.zeros(1, dtype=torch.float64, device="cuda"),
                    it=torch.zeros(1, dtype=torch.int32, device="cuda"),
                    st=torch.zeros(1, dtype=torch.int32, device="cuda"))

        def step():
            rlqr.rlqr_factor(dp, opts, ws, bufs["flags"], bufs["st"])
            rlqr.rlqr_solve(dp, opts, ws, bufs["x"], bufs["u"], bufs["y"], bufs["rel"],
                            bufs["it"], bufs["st"])
        return step, bufs

    def timed(step, steps, warmup):
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    step, bufs = make(rlqr.RLQR_MIXED, rlqr.RLQR_ALGO_SCAN)
    chunks = int((N + max(8, (N + 443) // 444) - 1) // max(8, (N + 443) // 444))
    tune = None
    if args.autotune:
        # the scan's tile (chunk count) chosen by timing the candidates; the
        # default chunking is timed beside it
        ms_default = timed(step, args.steps, args.warmup)
        o = rlqr.make_opts(rlqr.RLQR_MIXED, algo=rlqr.RLQR_ALGO_SCAN, tol=TOL, max_refine=3)
        wst = rlqr.alloc_workspace(rlqr.rlqr_workspace_bytes(N, n, m, o))
        chunks, tms = rlqr.rlqr_autotune_scan(dp, o, wst, bufs["x"], bufs["u"], bufs["y"],
                                              bufs["flags"])
        del wst
        tune = {"chunks": chunks, "autotune_ms": tms, "default_ms": ms_default,
                "candidates": list(rlqr.SCAN_CHUNK_CANDIDATES)}
    rlqr.rlqr_instrument(True)
    with ClockSampler(0) as clk:
        ms = timed(step, args.steps, args.warmup)
    report = rlqr.rlqr_instrument_report()
    rlqr.rlqr_instrument(False)
    rel = float(bufs["rel"].item())
    flags_gpu = bufs["flags"].cpu().numpy()
    step64, bufs64 = make(rlqr.RLQR_FP64, rlqr.RLQR_ALGO_SEQ)
    ms64 = timed(step64, fp64_reps, fp64_warmup)
    rel64 = None
    value = N / (ms / 1e3)
    # CPU baseline: the oracle on a bounded prefix of the horizon
    S = 4096
    sub = inputs.Problem(S, n, m, p.Q[:S + 1], p.M[:S], p.R[:S], p.q[:S + 1], p.r[:S], p.A[:S],
                         p.B[:S], p.c[:S + 1], p.delta)
    t0 = time.perf_counter()
    oracle.riccati(sub)
    cpu_s = time.perf_counter() - t0
    # roofline of the dominant kernel against the measured FP32 FMA rate (the
    # eliminations and solves of the scan run on the FP32 pipes), and the
    # fold's n x n products against a third of the measured TF32 mma rate
    # (they run as 3xTF32 mma.sync on the tensor pipe)
    pipes = rlqr.rlqr_measure_pipes()
    dom = max(report.items(), key=lambda kv: kv[1][1]) if report else None
    roof = None
    if dom is not None:
        name, (cnt, tot) = dom
        flops = scan_flops_per_stage(n, m).get(name)
        if flops:
            achieved = flops * N / (tot / cnt / 1e3) / 1e12
            roof = {"kernel": name, "bound": "fp32", "achieved": round(achieved, 3),
                    "peak": round(pipes["fp32x2_tflops"], 2), "unit": "TFLOP/s",
                    "frac": round(achieved / pipes["fp32x2_tflops"], 4),
                    "peak_source": "measured FP32 FMA rate (rlqr_measure_pipes)",
                    "flops_per_stage": flops, "launch_ms": round(tot / cnt, 4),
                    "share": round(tot / sum(v[1] for v in report.values()), 3), "traffic": None}
    roof_tc = None
    if "k_scan_reduce" in report and pipes.get("tf32_mma_tflops"):
        cnt, tot = report["k_scan_reduce"]
        prod = 10.0 * n ** 3  # the five n x n products of one combination per stage
        achieved = prod * N / (tot / cnt / 1e3) / 1e12
        peak = pipes["tf32_mma_tflops"] / 3.0
        roof_tc = {"kernel": "k_scan_reduce (its n x n products)", "bound": "tensor",
                   "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                   "frac": round(achieved / peak, 4),
                   "peak_source": "measured TF32 mma.sync rate (rlqr_measure_tf32) / 3 for 3xTF32",
                   "flops_per_stage": prod, "launch_ms": round(tot / cnt, 4)}
    line = {"metric": METRIC, "value": value, "unit": "stage-solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (FP32 scan; FP64 certificate, residual, correction)",
            "data": "synthetic",
            "config": {"workload": f"one dual-regularized LQR, n_x=32, n_u=8, N={N}, delta=1e-7, "
                                   "rho(A)=0.99, cond(Q)=cond(R)=1e4", "algo": "scan",
                       "chunks": chunks, "autotune": tune,
                       "l2": f"inputs {21.5e3 * N / 1e9:.2f} GB" + (
                           " > L2 (no flush needed)" if N >= 8192 else "")},
            "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in report.items()},
            "accuracy": {"rel_resid": rel, "all_le_tol": rel <= TOL,
                         "iters": int(bufs["it"].item()), "status": int(bufs["st"].item())},
            "fp64_plain_seq": {"value": N / (ms64 / 1e3), "ms_per_step": ms64,
                               "rel_resid": float(bufs64["rel"].item())},
            "speedup_vs_fp64_plain": ms64 / ms,
            "roofline": roof, "roofline_tensor": roof_tc,
            "cpu_baseline": {"value": S / cpu_s, "unit": "stage-solves/s", "cores": 1,
                             "kind": "oracle", "sample": f"the first {S} stages, {cpu_s:.2f} s"},
            "flags_all_pd": bool((flags_gpu == 3).all()),
            "clocks": clk.summary()}
    return line


def escalated_instances(ws, count):
    """Per instance of a batched solve: 1 if the FP64 recursion decided its
    pivot certificate (the escalated field, int32 at byte 56 of the
    instance's state; the instance offsets are the int64 array at the head
    of the batched workspace)."""
    import torch
    offs = ws[:8 * count].view(torch.int64)
    idx = offs.unsqueeze(1) + 56 + torch.arange(4, device=ws.device)
    return ws[idx].contiguous().view(torch.int32).reshape(count).cpu().numpy()


def _ragged_instance(arg):
    from paper_2509_16370_b300 import inputs
    b, (N, n, m) = arg
    return inputs.workload4_instance(b, N, n, m)


def run_ragged(args):
    print(json.dumps(measure_ragged(args, args.ragged, args.ragged_n)), flush=True)


def measure_ragged(args, count, only_n=0):
    """The first `count` instances of the ragged batch (N in 32..2048, n in
    {6, 12, 24, 48}, m = n/3): rlqr_solve_batched mixed vs plain FP64.
    Instances are generated by a process pool (spawn).  CPU baseline: the
    oracle's recursion on the batch's instances in order, one core, about
    5 s."""
    import multiprocessing as mp
    import torch
    import oracle
    from paper_2509_16370_b300 import inputs, rlqr
    items = list(enumerate(inputs.workload4_dims(4096)[:count]))
    if only_n:  # one size class of that sample
        items = [(b, d) for b, d in items if d[1] == only_n]
    dims = [d for _, d in items]
    with mp.get_context("spawn").Pool(min(32, os.cpu_count() or 1)) as pool:
        probs = pool.map(_ragged_instance, items, chunksize=4)
    db = rlqr.DeviceBatch.from_problems(probs)
    # CPU baseline sample: instances in batch order until ~5 s of oracle time
    cpu_stages, t0 = 0, time.perf_counter()
    for pb in probs:
        oracle.riccati(pb)
        cpu_stages += pb.N
        if time.perf_counter() - t0 >= 5.0:
            break
    cpu_s = time.perf_counter() - t0
    del probs  # the batch is on the device; at full size the host copy is ~76 GB
    stages = sum(N for N, _, _ in dims)
    data_gb = sum(8 * ((N + 1) * n * n + N * (2 * n * m + m * m + n * n) + (N + 1) * n * 2 + N * m)
                  for N, n, m in dims) / 1e9
    B = len(dims)

    def timed(prec, steps, warmup, instrument=False):
        opts = rlqr.make_opts(prec, tol=TOL, max_refine=6)
        ws = rlqr.alloc_workspace(rlqr.rlqr_batched_workspace_bytes(db, opts))
        st = torch.zeros(B, dtype=torch.int32, device="cuda")
        rel = torch.zeros(B, dtype=torch.float64, device="cuda")
        it = torch.zeros(B, dtype=torch.int32, device="cuda")
        for _ in range(warmup):
            rlqr.rlqr_solve_batched(db, opts, ws, st, rel, it)
        torch.cuda.synchronize()
        if instrument:
            rlqr.rlqr_instrument(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            rlqr.rlqr_solve_batched(db, opts, ws, st, rel, it)
        e1.record()
        torch.cuda.synchronize()
        report = rlqr.rlqr_instrument_report() if instrument else {}
        rlqr.rlqr_instrument(False)
        relv, stv = rel.cpu().numpy(), st.cpu().numpy()
        acc = dict(max_rel=float(relv.max()), all_le_tol=bool(np.all(relv <= TOL)),
                   max_iters=int(it.max().item()), statuses=sorted(set(stv.tolist())))
        if prec == rlqr.RLQR_MIXED:
            esc = escalated_instances(ws, B)
            acc["escalated"] = {f"n={nn}": int(sum(int(e) for e, (_, n_, _) in zip(esc, dims)
                                                   if n_ == nn))
                                for nn in sorted({d[1] for d in dims})}
            acc["escalated_stages"] = int(sum(N_ for e, (N_, _, _) in zip(esc, dims) if e))
        return e0.elapsed_time(e1) / steps, report, acc

    # setup, not timed: the autotuner times the mixed batch's sweep routes
    # (one launch per size class on concurrent streams / one persistent
    # launch) and records the faster one, which the timed solves then take
    tune = None
    o_t = rlqr.make_opts(rlqr.RLQR_MIXED, tol=TOL, max_refine=6)
    try:
        ws_t = rlqr.alloc_workspace(rlqr.rlqr_batched_workspace_bytes(db, o_t))
        route, tms = rlqr.rlqr_autotune_batched(db, o_t, ws_t)
        tune = {"sweep_route": {rlqr.SWEEP_ROUTE_STREAMS: "class streams",
                                rlqr.SWEEP_ROUTE_PERSISTENT: "persistent launch"}[route],
                "ms": round(tms, 3)}
        del ws_t
    except rlqr.RlqrError:
        tune = {"sweep_route": "class streams (sizes outside the persistent sweep)"}
    with ClockSampler(0) as clk:
        ms, report, acc = timed(rlqr.RLQR_MIXED, args.steps, args.warmup, True)
    ms64, _, acc64 = timed(rlqr.RLQR_FP64, max(1, args.steps // 4), 1)
    peaks = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    alg_bytes = sum(N * (8 * (2 * n * n + 2 * n * m + m * m + 2 * n + m) + 8 * (2 * n + m) + 1)
                    for N, n, m in dims)
    achieved = alg_bytes / (ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": stages / (ms / 1e3), "unit": "stage-solves/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (FP32 sweep; FP64 certificate, residual, correction)",
            "data": "synthetic",
            "config": {"workload": (f"the n={only_n} instances ({B}) of " if only_n
                                    else f"{B} instances: ") +
                                   f"the first {count} of the ragged batch of 4096 "
                                   "(N in 32..2048, n in {6,12,24,48}, m = n/3, barrier-scaled "
                                   "diagonals)", "instances": B, "stages": stages,
                       "data_gb": round(data_gb, 2), "autotune": tune},
            "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in report.items()},
            "roofline": {"kernel": "whole solve (size classes run concurrently)", "bound": "hbm",
                         "achieved": round(achieved, 2), "peak": hbm,
                         "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                         "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": None,
                         "algorithmic_bytes": alg_bytes},
            "accuracy": acc,
            "fp64_plain": {"value": stages / (ms64 / 1e3), "ms_per_step": ms64, **acc64},
            "speedup_vs_fp64_plain": ms64 / ms,
            "cpu_baseline": {"value": cpu_stages / cpu_s, "unit": "stage-solves/s", "cores": 1,
                             "kind": "oracle",
                             "sample": f"{cpu_stages} stages of the first instances, {cpu_s:.1f} s"},
            "clocks": clk.summary()}
    return line


def run_ours(args):
    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    from paper_2509_16370_b300 import inputs, rlqr

    bh = inputs.workload2()
    db = rlqr.DeviceBatch.from_uniform(bh)
    B, N, n, m = bh.count, bh.N, bh.n, bh.m
    stages = B * N
    stream = torch.cuda.current_stream()

    def setup(prec):
        opts = rlqr.make_opts(prec, tol=TOL, max_refine=3)
        ws = rlqr.alloc_workspace(rlqr.rlqr_batched_workspace_bytes(db, opts))
        st = torch.zeros(B, dtype=torch.int32, device="cuda")
        rel = torch.zeros(B, dtype=torch.float64, device="cuda")
        it = torch.zeros(B, dtype=torch.int32, device="cuda")
        return opts, ws, st, rel, it

    def timed(prec, steps, warmup, instrument=False):
        opts, ws, st, rel, it = setup(prec)
        for _ in range(warmup):
            rlqr.rlqr_solve_batched(db, opts, ws, st, rel, it)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if instrument:
            rlqr.rlqr_instrument(True)
        e0.record(stream)
        for _ in range(steps):
            rlqr.rlqr_solve_batched(db, opts, ws, st, rel, it)
        e1.record(stream)
        torch.cuda.synchronize()
        report = rlqr.rlqr_instrument_report() if instrument else {}
        if instrument:
            rlqr.rlqr_instrument(False)
        if world > 1:
            torch.distributed.barrier()
        ms = rank_max(e0.elapsed_time(e1) / steps, world)
        stv = st.cpu().numpy()
        relv = rel.cpu().numpy()
        ok = bool(np.all(relv <= TOL) and np.all((stv == 0) | (stv == 1)))
        esc = int(escalated_instances(ws, B).sum()) if prec == rlqr.RLQR_MIXED else 0
        return ms, report, dict(max_rel=float(relv.max()), ok=ok, iters=int(it.max().item()),
                                not_pd=int((stv == 1).sum()), escalated=esc)

    # the arithmetic pipes' measured rates (roofline denominators of the FP64
    # and FP32 kernels), taken before the timed regions
    pipes = rlqr.rlqr_measure_pipes()
    # setup, not timed: the autotuner times the batch's residual routes
    # (warp per instance / grid over all stages) and records the faster one
    # for this shape, which the timed solves then take
    tune = {}
    for prec, name in ((rlqr.RLQR_MIXED, "mixed"), (rlqr.RLQR_FP64, "fp64")):
        o_t, ws_t, st_t, _, _ = setup(prec)
        if args.residual_route:
            # a fixed route (profiling runs: timings under a profiler would
            # steer the tuner to another route than the plain bench takes)
            route = args.residual_route if prec == rlqr.RLQR_MIXED else rlqr.RES_ROUTE_WARP
            rlqr.rlqr_tune_batched_set(db, o_t, route)
            tms = None
        else:
            route, tms = rlqr.rlqr_autotune_batched(db, o_t, ws_t, st_t)
        tune[name] = {"residual_route": {rlqr.RES_ROUTE_WARP: "warp",
                                         rlqr.RES_ROUTE_GRID: "grid",
                                         rlqr.RES_ROUTE_FUSED: "fused into the first pass",
                                         rlqr.RES_ROUTE_WARP_DUO: "warp, two-warp refinement",
                                         rlqr.RES_ROUTE_FUSED_DUO:
                                             "fused into the first pass, two-warp refinement"}[route],
                      "ms": None if tms is None else round(tms, 4)}
        del ws_t
    with ClockSampler(local) as clk:
        ms_mixed, report, chk_mixed = timed(rlqr.RLQR_MIXED, args.steps, args.warmup, True)
    ms_fp64, report64, chk_fp64 = timed(rlqr.RLQR_FP64, max(3, args.steps // 4), args.warmup, True)

    # end to end through the C ABI from pinned host buffers: every step copies
    # its inputs in, solves and copies its solution, flags and backward
    # errors out.  Two batches are in flight -- step i uses buffer set i % 2
    # on its own stream -- so that one step's PCIe copies overlap the other
    # step's solve, as a stream of batches would be served.
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(bh, k)).reshape(-1)).pin_memory()
            for k in ("Q", "M", "R", "q", "r", "A", "B", "c")}
    slots = []
    for j in range(2):
        dbj = db if j == 0 else rlqr.DeviceBatch.from_uniform(bh)
        opts, ws, st, rel, it = setup(rlqr.RLQR_MIXED)
        slots.append(dict(db=dbj, opts=opts, ws=ws, st=st, rel=rel, it=it,
                          stream=torch.cuda.Stream(),
                          hx=torch.empty(dbj.x.numel(), dtype=torch.float64).pin_memory(),
                          hu=torch.empty(dbj.u.numel(), dtype=torch.float64).pin_memory(),
                          hy=torch.empty(dbj.y.numel(), dtype=torch.float64).pin_memory(),
                          hf=torch.empty(dbj.pivot_pd.numel(), dtype=torch.uint8).pin_memory(),
                          hrel=torch.empty(B, dtype=torch.float64).pin_memory()))
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = sum(slots[0][k].numel() * slots[0][k].element_size()
              for k in ("hx", "hu", "hy", "hf", "hrel"))

    def e2e_step(i):
        S = slots[i % 2]
        dbj = S["db"]
        with torch.cuda.stream(S["stream"]):
            for k, t in host.items():
                dbj.bufs[k].copy_(t, non_blocking=True)
            rlqr.rlqr_solve_batched(dbj, S["opts"], S["ws"], S["st"], S["rel"], S["it"])
            S["hx"].copy_(dbj.x, non_blocking=True)
            S["hu"].copy_(dbj.u, non_blocking=True)
            S["hy"].copy_(dbj.y, non_blocking=True)
            S["hf"].copy_(dbj.pivot_pd, non_blocking=True)
            S["hrel"].copy_(S["rel"], non_blocking=True)

    for i in range(args.warmup):
        e2e_step(i)
    torch.cuda.synchronize()
    e2e_steps = max(4, args.steps // 4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for S in slots:
        S["stream"].wait_stream(stream)
    for i in range(e2e_steps):
        e2e_step(i)
    for S in slots:
        stream.wait_stream(S["stream"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = rank_max(e0.elapsed_time(e1) / e2e_steps, world)
    e2e_ok = all(bool((S["hrel"] <= TOL).all()) for S in slots)

    if rank != 0:
        return
    value = job_rate(stages, world, ms_mixed)
    fp64_value = job_rate(stages, world, ms_fp64)
    launches = sum(c for c, _ in report.values())
    line = {
        "metric": METRIC, "value": value, "unit": "stage-solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_mixed,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 (FP32 sweep; FP64 certificate, residual, correction)",
        "data": "synthetic", "config": dict(WORKLOAD, parallelism=f"replicas x{world}",
                                              precision="mixed", max_refine=3, tol=TOL,
                                              autotune=tune),
        "roofline": roofline(report, args.steps, n, m, stages, load_peaks(), pipes["fp64_tflops"],
                             chain=(N, B, clk.summary().get("sm_mhz"))),
        "pipes": {k: round(v, 2) for k, v in pipes.items()},
        "kernels": {k: {"launches": c, "ms_total": round(t, 4)} for k, (c, t) in report.items()},
        "gpu_launches": launches,
        "accuracy": {"max_rel_resid": chk_mixed["max_rel"], "all_le_tol": chk_mixed["ok"],
                     "max_refine_iters": chk_mixed["iters"], "not_pd_instances": chk_mixed["not_pd"],
                     "escalated_instances": chk_mixed["escalated"]},
        "fp64_plain": {"value": fp64_value, "ms_per_step": ms_fp64,
                       "max_rel_resid": chk_fp64["max_rel"], "all_le_tol": chk_fp64["ok"],
                       "roofline": fp64_sweep_roofline(report64, n, m, stages, pipes),
                       # the plain recursion's own floor: its flops at the
                       # measured FP64 FMA rate (factor alone, no residual)
                       "fp64_pipe_floor_ms_per_step":
                           seq_flops_per_stage(n, m) * stages / (pipes["fp64_tflops"] * 1e12) * 1e3},
        "speedup_vs_fp64_plain": value / fp64_value,
        "speedup_vs_fp64_pipe_floor":
            seq_flops_per_stage(n, m) * stages / (pipes["fp64_tflops"] * 1e12) * 1e3 / ms_mixed,
        "e2e": {"value": job_rate(stages, world, ms_e2e), "unit": "stage-solves/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
                "batches_in_flight": 2, "all_le_tol": e2e_ok},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(bh, args.cpu_seconds)
    if world == 1 and not args.no_extras:
        # the other configurations of the metric, each with its own roofline
        # and CPU baseline (single GPU; the headline stays the batch above)
        del db, ws, host
        torch.cuda.empty_cache()
        extras = {}
        few = argparse.Namespace(**{**vars(args), "steps": 5, "warmup": 3})
        lat = argparse.Namespace(**{**vars(args), "steps": 50, "warmup": 5})
        ipm_args = argparse.Namespace(**{**vars(args), "steps": 1, "ipm": 8192,
                                         "cpu_seconds": min(args.cpu_seconds, 5.0)})
        for key, fn in (("latency", lambda: measure_latency(lat)),
                        ("long_horizon", lambda: measure_long_horizon(few, fp64_warmup=0)),
                        ("ragged", lambda: measure_ragged(few, 512)),
                        ("ipm", lambda: measure_ipm(ipm_args))):
            try:
                extras[key] = fn()
            except Exception as exc:  # reported, never hidden
                extras[key] = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.empty_cache()
        line["configs"] = extras
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 500 for the batch workload, so that the clock "
                         "sampler sees the timed region; 20 for the reference arm and "
                         "--latency, 3 for --ragged and --long-horizon)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations (small instance, long horizon, ragged)")
    ap.add_argument("--profile-instances", type=int, default=0,
                    help="profiling case: the mixed solve on the first K instances only")
    ap.add_argument("--autotune", action="store_true",
                    help="with --long-horizon: choose the scan's chunk count by timing first")
    ap.add_argument("--long-horizon", action="store_true",
                    help="the single long-horizon instance (associative scan)")
    ap.add_argument("--lh-stages", type=int, default=65536,
                    help="with --long-horizon: the horizon N (smaller for profiling)")
    ap.add_argument("--cross", type=int, default=0,
                    help="cross-stage variables: time rlqr_solve_cross with p = CROSS")
    ap.add_argument("--ipm", type=int, default=0,
                    help="the regularized IPM on the first IPM cart-double-pendulum instances")
    ap.add_argument("--ipm-study", type=int, default=0,
                    help="why cold IPM solves stop short, on the first K instances")
    ap.add_argument("--diag", action="store_true",
                    help="general diagonal Delta_i: rlqr_solve_diag beside the scalar-delta solve")
    ap.add_argument("--warm-start", type=int, default=0,
                    help="learned warm start: IPM runs for the training set (multiple of 8192)")
    ap.add_argument("--ws-steps", type=int, default=6000,
                    help="with --warm-start: Adam steps")
    ap.add_argument("--ipm-hessian", choices=["fp32", "fp64", "gn"], default="fp32",
                    help="with --ipm: the Hessian of the Lagrangian (exact in FP32 or FP64, or "
                         "Gauss-Newton)")
    ap.add_argument("--ipm-max-iter", type=int, default=0,
                    help="with --ipm: iteration limit (default 300; smaller for profiling)")
    ap.add_argument("--residual-route", type=int, default=0,
                    help="fix the batched residual route of the headline batch instead of "
                         "autotuning it (1 = warp residual; for profiler runs)")
    ap.add_argument("--latency", action="store_true",
                    help="latency of one factor + solve of the small single instance")
    ap.add_argument("--ragged", type=int, default=0,
                    help="the first K instances of the ragged batch")
    ap.add_argument("--ragged-n", type=int, default=0,
                    help="with --ragged: only the instances of that state dimension")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.steps is None:
        args.steps = (20 if args.impl == "reference" or args.latency or args.cross or args.diag else
                      3 if (args.ragged or args.long_horizon) else
                      1 if args.ipm else
                      1 if args.profile_instances else 500)
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_instances > 0:
        run_profile_case(args)
    elif args.long_horizon:
        run_long_horizon(args)
    elif args.latency:
        run_latency(args)
    elif args.cross:
        run_cross(args)
    elif args.ipm:
        run_ipm(args)
    elif args.ipm_study:
        run_ipm_study(args)
    elif args.warm_start:
        run_warm_start(args)
    elif args.diag:
        run_diag(args)
    elif args.ragged > 0:
        run_ragged(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
