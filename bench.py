#!/usr/bin/env python
"""Benchmark: cell-velocity updates per second of the half-range LB Couette
time step on the single-large-solve workload (Nx = 2048 stretched nodes,
2Qx x Qy = 32 x 20 velocities, delta in {0.1, 1, 10, 100}: four solves per
step, FP32 state with compensated moment sums), one JSON line on stdout.

A step is one TVD RK-3 step (three fused stage launches) of all four solves.
Timing: W untimed warm-up steps, then K steps timed with CUDA events on the
launching stream, an L2 flush (a 256 MiB write, not timed) between steps,
max over ranks. N > 1 runs N independent replicas (one batch per rank).
`--impl reference` times the FP64 CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-velocity updates/s"
FALLBACK_HBM_GBS = 6800.0
BYTES_PER_UPDATE_FP32 = 64   # 16 state values per cell-velocity step: each stage reads its input (and, after
                              # the first, the RK base) and writes its output, both fields: (2+3+3) x 2 values
BYTES_PER_UPDATE_FP64 = 128
# algorithmic FP64 operations of one cell-velocity update (both fields, three stages): per face
# and field the WENO-5 reconstruction (three candidate values 15, three smoothness indicators 36,
# epsilon 3, weights 9, normalisation 9: 72, a division counted as one operation), per node and
# field the relaxation to the Shakhov target and the RK combination (~20), per node the moment
# sums (~12): 2 (72 + 20) + 12 = 196 per stage
FLOPS_PER_UPDATE_FP64 = 3 * 196


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-steady", action="store_true", help="skip the steady-solves leg")
    ap.add_argument("--no-single", action="store_true", help="skip the single-solve leg")
    ap.add_argument("--no-persistent", action="store_true", help="skip the persistent-form leg")
    ap.add_argument("--form", choices=["auto", "cluster", "solo", "full", "split", "splitfull"], default="auto",
                    help="kernel form of the batched launch when --cluster fixes the shape (full: solo form "
                         "with 256-row chunks, cluster size following; split: a node-step launch per stage)")
    ap.add_argument("--cluster", type=int, default=0,
                    help="chunk CTAs per tile of the batched launch (0: autotune; fix it to profile a shape)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="state precision of the timed run (fp32: the headline path)")
    return ap.parse_args()


def workload_config():
    return {"workload": "single large solve: Nx=2048 tanh-stretched (spacing ratio 10), "
                        "HHLB(15;16)xHLB(19;20) = 640 velocities, delta in {0.1,1,10,100}, "
                        "u_w=+-0.1*sqrt(2kT/m), omega=0.66, Pr=2/3",
            "solves_per_step": 4, "Nx": 2048, "velocities": 640,
            "l2": "flushed between timed steps (256 MiB write)", "data": "synthetic"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if "Active" in val and "Not" not in val:
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        for k in ("hbm_gbs", "hbm_GBps", "hbm"):
            if k in d and isinstance(d[k], (int, float)):
                return float(d[k]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


def profiled_traffic(precision: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary,
    or None when the kernel source changed since the counters were taken."""
    import hashlib
    src = os.path.join(ROOT, "paper_1810_07803_gb300", "csrc", "lbc_kernels.cu")
    prof = os.path.join(ROOT, "profiles", f"stage_batch_kernel_{precision}_c2.md")
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        fields = dict(ln.split(":", 1) for ln in open(prof).read().splitlines() if ln.count(":") == 1
                      and ln.split(":", 1)[0].strip() in ("kernel_source_sha256_16", "traffic_bytes_per_launch"))
        if fields.get("kernel_source_sha256_16", "").strip() != digest:
            return None
        return float(fields["traffic_bytes_per_launch"]) if "traffic_bytes_per_launch" in fields else None
    except (OSError, ValueError):
        return None


def cpu_baseline(seconds_target=8.0):
    """The FP64 oracle as it stands, on the host cores, on bounded samples of the same
    workload: whole RK-3 steps of the delta = 1 solve, with the OpenMP build of the oracle
    on every core (the reported value) and with the plain build on one core; and the small
    configuration (Nx = 64, 8 x 4 velocities, FP64) run to r < 1e-10 on one core."""
    from oracle.oracle import Oracle
    from paper_1810_07803_gb300 import workloads
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    out = {}
    for parallel in (True, False):
        o = Oracle(workloads.c2(1.0, precision="fp64"), parallel=parallel)
        o.run(1)
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < seconds_target:
            o.run(1)
            n += 1
        dt = time.perf_counter() - t0
        out[parallel] = (o.V * o.Nx * n / dt, n)
    o = Oracle(workloads.c1())
    t0 = time.perf_counter()
    k, r = o.run_to_steady(1e-10, 200000)
    t1 = time.perf_counter() - t0
    return {"value": out[True][0], "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{out[True][1]} RK-3 steps of the delta=1 solve (Nx=2048, 640 velocities), FP64, "
                      f"OpenMP build of the oracle on {cores} threads",
            "single_core": {"value": out[False][0], "unit": METRIC, "cores": 1,
                            "sample": f"{out[False][1]} RK-3 steps of the same solve, plain build, 1 thread"},
            "small_config_to_steady": {"steps": k, "residual": r, "seconds": t1, "solves_per_s": 1.0 / t1,
                                       "cores": 1, "workload": "Nx=64 uniform, 8x4 velocities, delta=1, FP64, "
                                                               "rest start to r < 1e-10"}}


def steady_leg(n=64, fp64_sample=8, residual=1e-10, fp32_cap=100_000, stall_window=8192, seed=5):
    """Steady solves/s at equal moment error: n small Couette solves (the serving workload's
    draw) as one batch with the compensated FP32 state, against the plain form, FP64 single
    solves one after the other, on the first fp64_sample of them; both with local pseudo-time
    steps. Each arm's moments are compared with the limit (an FP64 batch of the same solves run
    to r < 1e-12, not timed). These solves contract by ~0.1 % per step, so the FP64 arm needs
    r < 1e-10 to come within 1e-5 of the limit; the FP32 evaluation of the right-hand side keeps
    the FP32 residual above ~1e-9, so each FP32 solve stops at r < 1e-10, at the stall rule (its
    residual has set no new low, by 1 %, for stall_window steps) or after fp32_cap steps,
    and its error against the limit is the measure. Completion time of a batched solve = batch
    time x its steps / the most steps (p50/p99 over the n)."""
    import numpy as np
    import torch
    from paper_1810_07803_gb300 import lbc, serve
    rng = np.random.default_rng(seed)
    reqs = [dict(serve.small_solve(rng), local_dt=1) for _ in range(n)]
    ref = lbc.Batch([dict(r, precision="fp64") for r in reqs], cluster=1)
    ref.run_to_steady(1e-12, 2_000_000, raise_notconv=False)
    limit = [ref.moments(i) for i in range(n)]
    ref.close()
    b = lbc.Batch([dict(r, precision="fp32", compensated=1) for r in reqs], cluster=1)
    b.set_stall_window(stall_window)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ks, rs = b.run_to_steady(residual, fp32_cap, raise_notconv=False)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    done = tb * np.asarray(ks, dtype=float) / max(ks)
    err32 = max(serve.moment_error(b.moments(i), limit[i]) for i in range(n))
    b.close()
    err64 = 0.0
    t64 = 0.0
    for i in range(fp64_sample):
        s = lbc.Solver(dict(reqs[i], precision="fp64"))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.run_to_steady(residual, 400_000)
        t64 += time.perf_counter() - t0
        err64 = max(err64, serve.moment_error(s.moments(), limit[i]))
        s.close()
    return {"metric": "steady solves/s", "batched_fp32": n / tb, "plain_fp64": fp64_sample / t64,
            "p50_s": float(np.percentile(done, 50)), "p99_s": float(np.percentile(done, 99)),
            "moment_error_batched_fp32": err32, "moment_error_plain_fp64": err64, "residual": residual,
            "fp32_steps_cap": fp32_cap, "fp32_at_cap": int(sum(k >= fp32_cap for k in ks)),
            "fp32_stall_window": stall_window,
            "fp32_stalled": int(sum(k < fp32_cap and r >= residual for k, r in zip(ks, rs))),
            "fp32_steps_p50_max": [float(np.percentile(ks, 50)), int(max(ks))],
            "reference": "each solve's FP64 steady state to r < 1e-12 (max over moments of the normalised error)",
            "workload": f"{n} small Couette solves (Nx 32-160, Qx, Qy 4-8, delta 0.3-3; seed {seed}), local steps; "
                        f"batched arm: compensated FP32 state; plain FP64 timed on {fp64_sample} of them"}


def run_reference(args, rank, budget_s=150.0):
    """The FP64 oracle as it stands on every host core (its OpenMP build), on the same
    workload and metric: a step is one RK-3 step of all four solves. If K steps of the
    whole workload would exceed the time budget, each timed step is a bounded sample of
    it (one solve, rotating) and the units follow the sample."""
    if rank != 0:
        return
    from oracle.oracle import Oracle
    from paper_1810_07803_gb300 import workloads
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    solves = [Oracle(workloads.c2(d, precision="fp64"), parallel=True) for d in workloads.C2_DELTAS]
    t0 = time.perf_counter()
    for o in solves:
        o.run(1)
    full_step = time.perf_counter() - t0
    per_step = 1 if full_step * (args.steps + args.warmup) > budget_s else len(solves)
    for k in range(max(0, args.warmup - 1)):
        for j in range(per_step):
            solves[(k * per_step + j) % 4].run(1)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        for j in range(per_step):
            solves[(k * per_step + j) % 4].run(1)
        times.append(time.perf_counter() - t0)
    ms = sum(times) / len(times) * 1e3
    value = per_step * solves[0].V * solves[0].Nx / (ms / 1e3)
    sample = ("each step: one RK-3 step of all four solves" if per_step == 4 else
              "each step: one RK-3 step of one of the four solves (rotating), the whole workload's step "
              "exceeding the time budget")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed steps; {sample}; OpenMP build of the oracle, "
                                       f"{cores} threads, FP64"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(values, device):
    """Element-wise max of per-rank timings (ms) over the process group, or the
    values themselves on a single rank: the job is as slow as its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_value(units_per_rank, world, ms_per_step):
    """Whole-job throughput: every rank's units over the slowest rank's step time."""
    return units_per_rank * world / (ms_per_step / 1e3)


def time_steps(solvers, steps, warmup, flush):
    """ms per step of single solvers stepped one after the other (L2 flushed between steps)."""
    import torch
    for _ in range(warmup):
        for s in solvers:
            s.step(1)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        evs[k][0].record()
        for s in solvers:
            s.step(1)
        evs[k][1].record()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


def time_batch(batch, steps, warmup, flush):
    """(ms per step, ms per stage launch) of a batch, L2 flushed between steps.
    Steps go through the plain stepping call (lbc_batch_step), each timed with events
    around it on the current stream (the batch's stream). A second pass of the same
    number of steps times every stage launch with the events the library records
    around each (lbc_batch_step_timed), for the roofline."""
    import torch
    batch.step(warmup)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        evs[k][0].record()
        batch.step(1)
        evs[k][1].record()
    torch.cuda.synchronize()
    stage_ms = 0.0
    for k in range(steps):
        flush.zero_()
        stage_ms += batch.step_timed(1)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps, stage_ms / (3 * steps)


def time_group(batch, steps, warmup, flush):
    """ms per step of a batch stepped one step at a time, L2 flushed between steps (CUDA events)."""
    import torch
    batch.step(warmup)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        evs[k][0].record()
        batch.step(1)
        evs[k][1].record()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


def persistent_leg(batch, units, steps, warmup, flush, uneven=True):
    """The persistent form (one cooperative launch per group of steps) against the per-stage
    launches on the benchmark's batch, and on the 512-solve uneven batch."""
    from paper_1810_07803_gb300 import lbc, workloads
    out = {}
    batch.set_persistent(True)
    ms = time_group(batch, steps, warmup, flush)
    batch.set_persistent(False)
    out["four_large_solves"] = {"value": units / (ms / 1e3), "unit": METRIC, "ms_per_step": ms}
    if uneven:
        b = lbc.Batch(workloads.c4())
        b.autotune(2)
        u4 = sum(b.V[i] * b.Nx[i] for i in range(b.n))
        ms_stage = time_group(b, 10, 2, flush)
        b.set_persistent(True)
        ms_pers = time_group(b, 10, 2, flush)
        b.close()
        out["uneven_512"] = {"unit": METRIC, "stage_launches": u4 / (ms_stage / 1e3), "persistent": u4 / (ms_pers / 1e3),
                             "ms_per_step_stage_launches": ms_stage, "ms_per_step_persistent": ms_pers,
                             "cell_velocities": u4}
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_1810_07803_gb300 import build, lbc, workloads
    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_1810_07803_gb300", "liblbc.so")):
        build.build()
    if world > 1:
        dist.barrier()

    params = [workloads.c2(d, precision=args.precision) for d in workloads.C2_DELTAS]
    batch = lbc.Batch(params, cluster=args.cluster)
    # cells per CTA: chosen by timing every feasible cluster size, unless fixed
    if args.cluster != 0 and args.form != "auto":
        batch.set_form({"cluster": 0, "solo": 1, "full": 2, "split": 3, "splitfull": 4}[args.form])
    cluster = batch.autotune(3) if args.cluster == 0 else batch.shape()[0]
    nsol = batch.n
    V, Nx = batch.V[0], batch.Nx[0]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, launch_ms = time_batch(batch, args.steps, args.warmup, flush)
    ms, launch_ms = max_over_ranks([ms, launch_ms], "cuda")
    units = nsol * V * Nx
    value = whole_job_value(units, world, ms)

    # end to end through the public API: host states in (pinned), host moments out, every step
    host_states = []
    for i in range(nsol):
        t = torch.empty((2, V, Nx), dtype=torch.float64, pin_memory=True)
        batch.get_state(i, out=t)
        host_states.append(t)
    e2e_steps = min(args.steps, 20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        batch.set_states(host_states)
        batch.step(1)
        batch.moments_all()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks([(time.perf_counter() - t0) / e2e_steps], "cuda")[0]
    h2d = sum(hs.numel() * hs.element_size() for hs in host_states)
    d2h = nsol * lbc.NMOM * Nx * 8

    fp64 = None
    if not args.no_fp64 and args.precision == "fp32":
        s64 = [lbc.Solver(workloads.c2(d, precision="fp64")) for d in workloads.C2_DELTAS]
        ms64 = time_steps(s64, max(3, args.steps // 10), 2, flush)
        rate64 = len(s64) * V * Nx * world / (ms64 / 1e3)
        peak64 = lbc.measure_fp64_peak()
        ach64 = FLOPS_PER_UPDATE_FP64 * rate64 / 1e12
        fp64 = {"value": rate64, "ms_per_step": ms64,
                "note": "same workload, FP64 state and arithmetic, one solve per launch, solves in sequence",
                "roofline": {"bound": "fp64", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s",
                             "frac": ach64 / peak64, "flops_per_update": FLOPS_PER_UPDATE_FP64,
                             "peak_kind": "measured (lbc_measure_fp64_peak: FP64 FMA chains on every SM)",
                             "hbm_frac": BYTES_PER_UPDATE_FP64 * rate64 / 1e9 / measured_hbm_peak()[0]}}
        for s in s64:
            s.close()

    # the single-solve path: one solve (delta = 1) through the single-instance stage kernel
    single = None
    if not args.no_single:
        one = lbc.Batch([workloads.c2(1.0, precision=args.precision)])
        one.autotune(3)
        ms1, launch1 = time_batch(one, max(3, min(args.steps, 200)), args.warmup, flush)
        units1 = V * Nx
        peak1, _ = measured_hbm_peak()
        ach1 = BYTES_PER_UPDATE_FP32 * units1 / 3 / (launch1 / 1e3) / 1e9 if args.precision == "fp32" else \
            BYTES_PER_UPDATE_FP64 * units1 / 3 / (launch1 / 1e3) / 1e9
        single = {"value": units1 * world / (ms1 / 1e3), "unit": METRIC, "ms_per_step": ms1, "launch_ms": launch1,
                  "cluster": one.shape()[0], "kernel": "stage_kernel (single instance, descriptor as a parameter)",
                  "roofline": {"bound": "hbm", "achieved": ach1, "peak": peak1, "unit": "GB/s", "frac": ach1 / peak1},
                  "workload": "the delta=1 solve alone (Nx=2048, 640 velocities) through lbc_step's kernel"}
        one.close()

    persistent = None
    if not args.no_persistent:
        persistent = persistent_leg(batch, units, max(3, min(args.steps, 200)), args.warmup, flush,
                                    uneven=args.precision == "fp32")

    steady = None
    if not args.no_steady and args.precision == "fp32":
        steady = steady_leg()

    peak, peak_kind = measured_hbm_peak()
    launches_per_step = 4   # one batched launch per RK stage (all solves) and the step-counter bump
    bpu = BYTES_PER_UPDATE_FP32 if args.precision == "fp32" else BYTES_PER_UPDATE_FP64
    bytes_per_launch = bpu * units / 3   # one RK stage of every solve
    achieved = bytes_per_launch / (launch_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": workload_config(),
        "launch": {"cluster": cluster, "form": "one batched stage launch per RK stage for the four solves",
                   "kernel_form": batch.FORMS[batch.form], "state": args.precision},
        "e2e": {"value": units * world / e2e_s, "unit": METRIC, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "path": "per step: lbc_batch_set_states(pinned host f64, every solve) + lbc_batch_step(1) + "
                        "lbc_batch_moments_all(host)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": profiled_traffic(args.precision),
                     "kernel": "stage_batch_kernel<float>" if args.precision == "fp32" else "stage_batch_kernel<double>",
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bytes_per_launch,
                     "launch_ms": launch_ms},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    if single:
        line["single"] = single
    if persistent:
        line["persistent"] = persistent
    if fp64:
        line["fp64_plain"] = fp64
    if steady:
        line["steady"] = steady
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    batch.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
