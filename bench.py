#!/usr/bin/env python3
"""Benchmark of the correlated-pair hot path on one GB300.

Workload (a "step"): one full multilevel estimate of the periodic problem for
each eps in {1, 0.1, 1e-3} -- density 1 + cos(2 pi x) on [0, 1), T = 1,
dt0 = 0.5, M = 2, L = min(12, ceil(log2(dt0/(eps^2/4)))), QoI int x^2 f plus a
128-bin density -- with the sample counts N_l that the variance-optimal rule
gives for RMSE 1e-3 (fixed by one untimed adaptive pilot).  Every level of
every eps runs the pair kernel, the fixed-order finalize and the FP64
controller.

Metric: correlated particle-substeps (executed fine + coarse KD events) per
second.  `value` is timed on the device with CUDA events; `e2e` is the host
wall time of the same public calls (mlkd_estimate with host problem/result).
`--impl reference` times the CPU oracle on a bounded sample of the workload.
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

import workloads as W  # noqa: E402

METRIC = "correlated particle-substeps/s (fine+coarse KD events, periodic full MLMC, tol 1e-3)"
UNIT = "events/s"
EPS_SET = W.PERIODIC_EPS
TOL = 1e-3

# Algorithmic instruction budget per KD event of the FP32 pair kernel (lane
# instructions): Philox4x32-10 block, three uniforms, Box-Muller and -log u,
# the KD coefficients and position update, the aggregation weights.  Stated
# with its derivation in the design notes; the ncu summary
# profiles/pair_kernel_fp32_periodic.md gives the measured count.
INST_PER_FINE_EVENT = 190.0
INST_PER_COARSE_EVENT = 50.0
SMSP_PER_SM = 4
LANES = 32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32comp", "fp64"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def problems_for_rank(rank: int):
    """Each rank runs its own independent copy of the workload (its own
    Philox request ids): weak scaling, no data-path exchange."""
    return [W.periodic_problem(eps, seed=0, tol=TOL) | {"request": rank * 16 + i}
            for i, eps in enumerate(EPS_SET)]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

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
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, flag in zip(names, parts[4:8]):
                if flag.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2004_04071_gb300 as mk

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    prec = {"fp32": mk.PREC_FP32_DY64, "fp32comp": mk.PREC_FP32_COMP, "fp64": mk.PREC_FP64}[args.precision]
    ctx = mk.Context(local)
    stream = torch.cuda.current_stream()

    # ---- untimed pilot: N_l from the variance-optimal rule at tol 1e-3 ----
    probs = problems_for_rank(rank)
    fixed = []
    for d in probs:
        p = mk.make_problem(precision=prec, **{k: v for k, v in d.items()})
        r = ctx.estimate(p)
        fixed.append([lv["n"] for lv in r.levels])
    step_problems = [mk.make_problem(precision=prec, n_fixed=n, **d) for d, n in zip(probs, fixed)]

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda:%d" % local)

    def step():
        events = 0
        for p in step_problems:
            r = ctx.estimate(p, stream)
            events += sum(lv["events_f"] + lv["events_c"] for lv in r.levels)
        return events

    for _ in range(args.warmup):
        step()
    ctx.set_timing(True)
    ctx.get_timing(reset=True)

    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    dev_ms, host_s, events_total = 0.0, 0.0, 0
    for _ in range(args.steps):
        flush.zero_()                       # L2 flush outside the timed window
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        h0 = time.perf_counter()
        e0.record(stream)
        events_total += step()
        e1.record(stream)
        torch.cuda.synchronize()
        host_s += time.perf_counter() - h0
        dev_ms += e0.elapsed_time(e1)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    timing = ctx.get_timing(reset=True)

    # max over ranks of the timed region; sum of the work
    t_dev = dev_ms / 1e3
    t_host = host_s
    ev = float(events_total)
    if world > 1:
        t = torch.tensor([t_dev, t_host], dtype=torch.float64, device="cuda:%d" % local)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e = torch.tensor([ev], dtype=torch.float64, device="cuda:%d" % local)
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
        t_dev, t_host, ev = float(t[0]), float(t[1]), float(e[0])

    # events split for the roofline of the pair kernel (rank-local)
    fine = coarse = 0
    for p in step_problems:
        r = ctx.estimate(p)
        fine += sum(lv["events_f"] for lv in r.levels)
        coarse += sum(lv["events_c"] for lv in r.levels)
    launches_per_step = timing["launches"] / max(1, args.steps)
    kernel_s = timing["pair_kernel_ms"] / 1e3
    algo_inst = (fine * INST_PER_FINE_EVENT + coarse * INST_PER_COARSE_EVENT) * args.steps
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clocks.get("sm_mhz") or 1470.0
    peak = sm_count * SMSP_PER_SM * LANES * mhz * 1e6
    achieved = algo_inst / kernel_s if kernel_s > 0 else 0.0

    out = {
        "metric": METRIC, "value": ev / t_dev, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp32comp": "f32", "fp64": "f64"}[args.precision],
        "data": "synthetic (Philox streams; analytic homogeneous background)",
        "config": {"workload": "periodic full MLMC, eps in {1,0.1,1e-3}, T=1, dt0=0.5, M=2, "
                               "L=min(12,ceil(log2(dt0/(eps^2/4)))), tol=1e-3, 128 bins",
                   "precision": args.precision, "n_fixed": fixed,
                   "events_per_step": ev / args.steps / world,
                   "l2": "flushed (256 MB write) between timed steps; no input arrays"},
        "e2e": {"value": ev / t_host, "unit": UNIT,
                "h2d_bytes_per_step": len(step_problems) * (88 + 8 * 13),
                "d2h_bytes_per_step": len(step_problems) * (1400 + 8 * 128)},
        "gpu_launches": int(timing["launches"] + timing["other_launches"]),
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9,
                     "unit": "Ginst/s (lane instructions)",
                     "frac": achieved / peak if peak else None, "traffic": None,
                     "kernel": "pair_kernel<float, FP32_DY64, coupled>",
                     "launches_per_step": launches_per_step,
                     "avg_launch_ms": timing["pair_kernel_ms"] / max(1, timing["launches"]),
                     "peak_basis": "152 SM x 4 SMSP x 32 lanes x median SM clock under load"},
        "clocks": clocks,
    }
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds, fixed)
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def oracle_sample(cpu_seconds: float, fixed=None):
    """Times the oracle on a bounded sample of the workload.  Each round runs,
    for every eps and level, a slice of pairs proportional to that level's
    N_l (at least 32), continuing the pair index where the last round
    stopped; rounds repeat until about `cpu_seconds` have passed, on all host
    cores."""
    import oracle as O
    threads = os.cpu_count() or 1
    if fixed is None:
        fixed = [[max(100, 2 ** (12 - l)) for l in range(W.periodic_levels(e) + 1)] for e in EPS_SET]
    total = float(sum(sum(n) for n in fixed))
    per_round = 2e5                                   # pairs per round over all levels
    probs = []
    for eps, n_l in zip(EPS_SET, fixed):
        d = W.periodic_problem(eps)
        p = O.Problem(**{k: d[k] for k in ("eps", "T", "dt0", "M", "L", "qoi", "init", "nbins",
                                           "lo", "hi", "seed")})
        probs.append((p, [max(32, int(per_round * n / total)) for n in n_l]))
    nxt = [[0] * len(c) for _, c in probs]
    ev, rounds, t0 = 0, 0, time.perf_counter()
    while True:
        for j, (p, counts) in enumerate(probs):
            for level, cnt in enumerate(counts):
                s = O.run_level(p, level, nxt[j][level], cnt, threads=threads)
                nxt[j][level] += cnt
                ev += s.events_f + s.events_c
        rounds += 1
        dt = time.perf_counter() - t0
        if dt >= cpu_seconds:
            break
    pairs = sum(sum(x) for x in nxt)
    return {"value": ev / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d rounds over every eps and level of the workload, pairs per level "
                      "proportional to N_l (>= 32): %d pairs, %d events in %.1f s"
                      % (rounds, pairs, ev, dt)}


def cpu_baseline(cpu_seconds, fixed):
    try:
        return oracle_sample(cpu_seconds, fixed)
    except Exception as exc:  # the baseline must not sink the GPU line
        return {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                "sample": "failed: %s" % exc}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    per_step = max(1.0, min(15.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(per_step / 4)
    vals, evs, secs = [], 0, 0.0
    last = None
    for _ in range(args.steps):
        last = oracle_sample(per_step)
        vals.append(last["value"])
    value = statistics.mean(vals)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (Philox streams; analytic homogeneous background)",
           "config": {"workload": "periodic full MLMC, eps in {1,0.1,1e-3}, T=1, dt0=0.5, M=2, "
                                  "tol=1e-3, 128 bins (bounded sample per step)"},
           "impl": "reference",
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                            "sample": last["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
