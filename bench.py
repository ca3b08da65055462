#!/usr/bin/env python3
"""Benchmark of the correlated-pair hot path on one GB300.

Workload (a "step"): one full multilevel estimate of the periodic problem for
each eps in {1, 0.1, 1e-3} -- density 1 + cos(2 pi x) on [0, 1), T = 1,
dt0 = 0.5, M = 2, L = min(12, ceil(log2(dt0/(eps^2/4)))), QoI int x^2 f plus a
128-bin density -- with the sample counts N_l that the variance-optimal rule
gives for RMSE 1e-3 (fixed by one untimed adaptive pilot).  By default the
three estimates run together in the batched form (one persistent pair kernel
over a device work queue, scheduler and FP64 controller on the device, one
CUDA graph per step) with the autotuned pairs-per-thread and
substeps-per-launch; --form plain runs each level as its own launch.

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
    ap.add_argument("--precision", default="fp32comp", choices=["fp32", "fp32comp", "fp64"])
    ap.add_argument("--form", default="batch", choices=["batch", "plain"],
                    help="batched persistent form (default) or the per-level form")
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
    base_cfg = mk.batch_config(pairs_per_thread=1, substeps_per_launch=256, use_graph=1,
                               max_requests=16, max_nbins=128)
    ctx = mk.Context(local, arena_bytes=mk.batch_workspace_bytes(base_cfg))
    stream = torch.cuda.current_stream()
    dev = "cuda:%d" % local

    # ---- untimed: N_l from the variance-optimal rule at tol 1e-3, and the
    # time to tolerance of the adaptive estimate in this form -------------
    dicts = problems_for_rank(rank)
    adaptive = [mk.make_problem(precision=prec, **d) for d in dicts]
    t0 = time.perf_counter()
    if args.form == "batch":
        pilot = ctx.estimate_batch(adaptive, base_cfg)
    else:
        pilot = [ctx.estimate(p) for p in adaptive]
    ttt_first = time.perf_counter() - t0
    fixed = [[lv["n"] for lv in r.levels] for r in pilot]
    step_problems = [mk.make_problem(precision=prec, n_fixed=n, **d) for d, n in zip(dicts, fixed)]

    cfg = base_cfg
    tune = None
    if args.form == "batch" and prec != mk.PREC_FP64:
        cfg, secs = ctx.autotune_batch(step_problems, base_cfg)
        tune = {"best": cfg.as_dict(), "seconds_ppt_major": secs}

    def step():
        if args.form == "batch":
            rs = ctx.estimate_batch(step_problems, cfg, stream)
        else:
            rs = [ctx.estimate(p, stream) for p in step_problems]
        return sum(lv["events_f"] + lv["events_c"] for r in rs for lv in r.levels), rs

    # time to tolerance (adaptive, after warm-up of the code paths)
    def ttt_once(problems):
        t = time.perf_counter()
        if args.form == "batch":
            rs = ctx.estimate_batch(problems, cfg, stream)
        else:
            rs = [ctx.estimate(p, stream) for p in problems]
        return time.perf_counter() - t, rs

    for _ in range(args.warmup):
        step()
    ttt = sorted(ttt_once(adaptive)[0] for _ in range(3))[1]

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    ctx.get_timing(reset=True)
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    dev_ms, host_s, events_total = 0.0, 0.0, 0
    last = None
    for _ in range(args.steps):
        flush.zero_()                       # L2 flush outside the timed window
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        h0 = time.perf_counter()
        e0.record(stream)
        ev, last = step()
        events_total += ev
        e1.record(stream)
        torch.cuda.synchronize()
        host_s += time.perf_counter() - h0
        dev_ms += e0.elapsed_time(e1)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    timing = ctx.get_timing(reset=True)

    # roofline pass: the same step with the pair kernel timed per launch
    # (batched form in its host-loop variant, per-level form as it is)
    ctx.set_timing(True)
    ctx.get_timing(reset=True)
    fine = coarse = 0
    rsteps = max(1, min(args.steps, 10))
    for _ in range(rsteps):
        if args.form == "batch":
            hl = mk.batch_config(**dict(cfg.as_dict(), use_graph=0))
            rs = ctx.estimate_batch(step_problems, hl, stream)
        else:
            rs = [ctx.estimate(p, stream) for p in step_problems]
        fine += sum(lv["events_f"] for r in rs for lv in r.levels)
        coarse += sum(lv["events_c"] for r in rs for lv in r.levels)
    rt = ctx.get_timing(reset=True)
    ctx.set_timing(False)

    t_dev = dev_ms / 1e3
    t_host = host_s
    ev = float(events_total)
    if world > 1:
        t = torch.tensor([t_dev, t_host], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e = torch.tensor([ev], dtype=torch.float64, device=dev)
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
        t_dev, t_host, ev = float(t[0]), float(t[1]), float(e[0])

    kernel_s = rt["pair_kernel_ms"] / 1e3
    algo_inst = fine * INST_PER_FINE_EVENT + coarse * INST_PER_COARSE_EVENT
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clocks.get("sm_mhz") or 1470.0
    peak = sm_count * SMSP_PER_SM * LANES * mhz * 1e6
    achieved = algo_inst / kernel_s if kernel_s > 0 else 0.0
    kname = ("batch_pair_kernel" if args.form == "batch" else "pair_kernel") + \
        {"fp32": "<float, FP32_DY64>", "fp32comp": "<float, FP32_COMP>", "fp64": "<double, FP64>"}[args.precision]

    out = {
        "metric": METRIC, "value": ev / t_dev, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp32comp": "f32", "fp64": "f64"}[args.precision],
        "data": "synthetic (Philox streams; analytic homogeneous background)",
        "config": {"workload": "periodic full MLMC, eps in {1,0.1,1e-3}, T=1, dt0=0.5, M=2, "
                               "L=min(12,ceil(log2(dt0/(eps^2/4)))), tol=1e-3, 128 bins",
                   "form": args.form, "precision": args.precision, "n_fixed": fixed,
                   "batch_config": cfg.as_dict() if args.form == "batch" else None,
                   "autotune": tune,  # seconds over ppt {1,2,4,8} x substeps {16,64,256,unbounded}
                   "events_per_step": ev / args.steps / world,
                   "time_to_tolerance_s": ttt, "time_to_tolerance_first_call_s": ttt_first,
                   "estimates": [r.estimate for r in last],
                   "variances": [r.variance for r in last],
                   "l2": "flushed (256 MB write) between timed steps; no input arrays"},
        "e2e": {"value": ev / t_host, "unit": UNIT,
                "h2d_bytes_per_step": len(step_problems) * (88 + 8 * 13),
                "d2h_bytes_per_step": len(step_problems) * (1400 + 8 * 128)},
        "gpu_launches": int(timing["launches"] + timing["other_launches"]),
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9,
                     "unit": "Ginst/s (lane instructions)",
                     "frac": achieved / peak if peak else None, "traffic": None,
                     "kernel": kname,
                     "launches_timed": rt["launches"],
                     "avg_launch_ms": rt["pair_kernel_ms"] / max(1, rt["launches"]),
                     "events_timed": fine + coarse,
                     "peak_basis": "SMs x 4 SMSP x 32 lanes x median SM clock under load "
                                   "(issue-slot bound; algorithmic 190 lane-inst per fine event, "
                                   "50 per coarse event)"},
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
