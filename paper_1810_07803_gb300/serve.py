"""Serving loop on the instance pool: Couette solves arrive over time, are
admitted as device memory allows, run together (continuous batching) until each
reaches the steady-state residual, and leave; latency is arrival to result.

The pool (include/lbc.h, lbc_pool_*) steps every resident instance in one
batched launch per RK stage, and each instance stops at its own converged
step, so requests that arrive while others run join the next chunk of steps.
The plain comparison serves the same requests one at a time with a
single-instance FP64 solver.

    python -m paper_1810_07803_gb300.serve --rates 10,100,1000 --duration 10
"""
from __future__ import annotations

import argparse
import collections
import json
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import lbc

SQ2 = math.sqrt(2.0)


@dataclass
class Request:
    rid: int
    arrival: float                  # seconds after the start of the trace
    params: dict
    admitted: float | None = None
    finished: float | None = None
    steps: int = 0
    residual: float = math.inf
    converged: bool = False
    moments: np.ndarray | None = field(default=None, repr=False)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process of `rate` per second over [0, duration)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return np.array(out)
        out.append(t)


def small_solve(rng: np.random.Generator) -> dict:
    """One request of the served workload: a small Couette solve (Nx 32-160,
    Qx, Qy 4-8, delta log-U[0.3, 3], wall temperature ratio log-U[1, 2],
    u_w U[0.01, 0.3] sqrt(2kT/m), omega 0.66, Pr 2/3, wall-clustered grid)."""
    ratio = float(math.exp(rng.uniform(0.0, math.log(2.0))))
    TL = 2.0 / (1.0 + ratio)
    uw = float(rng.uniform(0.01, 0.3)) * SQ2
    return dict(delta=float(math.exp(rng.uniform(math.log(0.3), math.log(3.0)))), u_left=-uw, u_right=uw,
                T_left=TL, T_right=ratio * TL, Pr=2.0 / 3.0, omega=0.66, Nx=int(rng.integers(32, 161)),
                stretch_A=math.sqrt(0.9), Qx=int(rng.integers(4, 9)), Qy=int(rng.integers(4, 9)))


def make_trace(rate: float, duration: float, seed: int, draw=small_solve, **extra) -> list[Request]:
    """Requests of a Poisson trace; `extra` parameters (e.g. local_dt=1) go into every request."""
    times = poisson_arrivals(rate, duration, seed)
    rng = np.random.default_rng(seed + 1)
    return [Request(k, float(t), dict(draw(rng), **extra)) for k, t in enumerate(times)]


class Server:
    """Continuous batching on one GPU: FIFO admission by device footprint, chunks
    of `chunk` steps for all resident requests, retirement at convergence.

    clock: "wall" serves the trace in real time (latency in seconds); "steps"
    advances a virtual clock by one unit per step chunk, which makes admission
    order deterministic for tests.
    """

    def __init__(self, cluster: int = 1, precision: str = "fp32", budget_bytes: int = 16 << 30,
                 residual: float = 1e-8, chunk: int = 32, max_steps: int = 200_000,
                 max_instances: int = 4096, pool=None):
        # `pool` replaces the device pool (same methods as lbc.Pool), e.g. to test the scheduling
        self.pool = pool if pool is not None else lbc.Pool(cluster, precision, budget_bytes,
                                                           max_instances=max_instances, max_tiles=1 << 18)
        self.residual, self.chunk, self.max_steps = residual, chunk, max_steps

    def close(self):
        self.pool.close()

    def serve(self, requests: list[Request], clock: str = "wall") -> list[Request]:
        reqs = sorted(requests, key=lambda r: r.arrival)
        queue: collections.deque = collections.deque()
        active: dict[int, Request] = {}
        nxt = 0
        t0 = time.perf_counter()
        vclock = 0.0

        def now():
            return time.perf_counter() - t0 if clock == "wall" else vclock

        while nxt < len(reqs) or queue or active:
            t = now()
            while nxt < len(reqs) and reqs[nxt].arrival <= t:
                queue.append(reqs[nxt])
                nxt += 1
            while queue:                                   # FIFO admission while memory allows
                slot = self.pool.try_add(queue[0].params)
                if slot is None:
                    if not active:
                        raise RuntimeError("request larger than the pool budget")
                    break
                r = queue.popleft()
                r.admitted = t
                active[slot] = r
            if not active:                                 # idle until the next arrival
                if clock == "wall":
                    time.sleep(max(0.0, reqs[nxt].arrival - now()))
                else:
                    vclock = reqs[nxt].arrival
                continue
            done = set(self.pool.run(self.residual, self.chunk))
            vclock += 1.0
            t = now()
            for slot, r in list(active.items()):
                # an instance that did not converge in this chunk took all of its steps, so
                # its count is kept here; the pool is asked only about those that leave
                if slot not in done:
                    r.steps += self.chunk
                    if r.steps < self.max_steps:
                        continue
                _, _, _, steps, res = self.pool.info(slot)
                r.finished, r.steps, r.residual = t, steps, res
                r.converged = slot in done
                r.moments = self.pool.moments(slot)
                self.pool.remove(slot)
                del active[slot]
        return reqs


def serve_sequential_fp64(requests: list[Request], residual: float = 1e-8, max_steps: int = 200_000,
                          measure: int = 0) -> list[Request]:
    """The plain comparison: one request at a time, single-instance FP64 solver, in
    arrival order (a single FIFO server). measure = 0: every request is solved in real
    time (the server idles until the next arrival; latency = arrival to result).
    measure = k > 0: only the first k requests are solved and timed, and the queue of
    the whole trace is played with those service times in turn (start = max(arrival,
    previous finish)), for traces whose FP64 solves would take too long to run."""
    reqs = sorted(requests, key=lambda r: r.arrival)

    def solve(r: Request) -> None:
        s = lbc.Solver(dict(r.params, precision="fp64"))
        try:
            r.steps, r.residual = s.run_to_steady(residual, max_steps)
            r.converged = True
        except lbc.LbcError as e:
            if e.status != lbc.ENOTCONV:
                raise
            r.steps, r.residual = s.steps, math.inf
        r.moments = s.moments()
        s.close()

    if measure <= 0:
        t0 = time.perf_counter()
        for r in reqs:
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            r.admitted = time.perf_counter() - t0
            solve(r)
            r.finished = time.perf_counter() - t0
        return reqs
    service = []
    for r in reqs[:measure]:
        t1 = time.perf_counter()
        solve(r)
        service.append(time.perf_counter() - t1)
    free = 0.0
    for k, r in enumerate(reqs):
        r.admitted = max(r.arrival, free)
        r.finished = free = r.admitted + service[k % len(service)]
        if k >= measure:
            r.converged, r.steps = True, reqs[k % measure].steps
    return reqs


def moment_error(m: np.ndarray, ref: np.ndarray) -> float:
    """max over moments k of max_s |m_k - ref_k| / max(max_s |ref_k|, floor_k): floor 1 for
    n, T and the pressures, 1e-2 for velocities, shear stress and heat flux."""
    floors = np.array([1.0, 1e-2, 1e-2, 1.0, 1.0, 1.0, 1.0, 1e-2, 1e-2, 1e-2])
    scale = np.maximum(np.max(np.abs(ref), axis=1), floors)
    return float(np.max(np.max(np.abs(m - ref), axis=1) / scale))


def summary(reqs: list[Request], label: str, rate: float, duration: float) -> dict:
    lat = np.array([r.latency for r in reqs])
    span = max(r.finished for r in reqs) if reqs else 0.0
    ok = sum(r.converged for r in reqs)
    return {"server": label, "rate_per_s": rate, "duration_s": duration, "requests": len(reqs),
            "converged": ok, "solves_per_s": ok / span if span > 0 else 0.0,
            "latency_p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "latency_p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_steps": float(np.mean([r.steps for r in reqs])) if reqs else 0.0}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--rates", default="10,100,1000")
    ap.add_argument("--duration", type=float, default=10.0)
    ap.add_argument("--residual", type=float, default=1e-8)
    ap.add_argument("--cluster", type=int, default=1,
                    help="chunk CTAs per tile; 1 suits the small served requests (<= 256 velocities): more "
                         "CTAs per tile add per-CTA overhead and measured lower solves/s")
    ap.add_argument("--chunk", type=int, default=32)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--local-dt", action="store_true", help="local pseudo-time steps in both servers")
    ap.add_argument("--compensated", action="store_true", help="compensated FP32 state in the pool")
    ap.add_argument("--sequential-measure", type=int, default=0,
                    help="0: the FP64 sequential comparison solves every request in real time; k > 0: it solves "
                         "and times the first k and queues the rest with those service times")
    ap.add_argument("--no-sequential", action="store_true", help="serve with the pool only")
    args = ap.parse_args()
    extra = dict(local_dt=1) if args.local_dt else {}
    for rate in (float(x) for x in args.rates.split(",")):
        trace = make_trace(rate, args.duration, args.seed,
                           **dict(extra, **(dict(compensated=1) if args.compensated else {})))
        srv = Server(cluster=args.cluster, residual=args.residual, chunk=args.chunk)
        served = srv.serve(trace)
        out = summary(served, "pool-fp32", rate, args.duration)
        srv.close()
        out["local_dt"], out["compensated"] = bool(args.local_dt), bool(args.compensated)
        if args.no_sequential:
            print(json.dumps(out), flush=True)
            continue
        seq = make_trace(rate, args.duration, args.seed, **extra)
        seq_out = serve_sequential_fp64(seq, args.residual, measure=args.sequential_measure)
        # moment error of the pool's FP32 results against the FP64 solves of the same requests
        solved = seq_out if args.sequential_measure <= 0 else seq_out[:args.sequential_measure]
        errs = [moment_error(r.moments, q.moments) for r, q in zip(served, solved)]
        out["moment_error_vs_fp64"] = max(errs) if errs else None
        print(json.dumps(out), flush=True)
        out = summary(seq_out, "sequential-fp64", rate, args.duration)
        out["timing"] = ("every request solved in real time" if args.sequential_measure <= 0 else
                         f"{args.sequential_measure} solves measured, FIFO queue played with their service times")
        out["local_dt"] = bool(args.local_dt)
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
