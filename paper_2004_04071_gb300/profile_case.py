"""Small, fixed pair-kernel launches for profiling with ncu.

    python -m paper_2004_04071_gb300.profile_case [--precision fp32|fp32comp|fp64]
    python -m paper_2004_04071_gb300.profile_case --form batch

Per-level form: three launches of the pair kernel on cuda:0, each over 2^20
pairs (2^22 for the level-0 case), on the periodic problem of the benchmark:
  1. eps = 0.1, level 8  (mixed regime, R dt = 0.2)
  2. eps = 1e-3, level 6 (deep diffusive, one event per fine step)
  3. eps = 0.1, level 0  (initialisation-dominated, two events per path)
Device memory held: the 0.7 MB context arena.

Batched form: the benchmark's three periodic estimates (eps = 1, 0.1, 1e-3)
with fixed sample counts scaled by 1/8 (by 2^scale / 8 with --scale) in one
batched call with unbounded slices and no graph, so that the pair work is one
batch_pair_kernel launch.  Device memory held: the batch arena (about 0.3 GB)
at any scale.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import paper_2004_04071_gb300 as mk
    import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32comp", "fp64"])
    ap.add_argument("--scale", type=int, default=0, help="log2 extra scale of the pair counts")
    ap.add_argument("--form", default="level", choices=["level", "batch"])
    a = ap.parse_args()
    prec = {"fp32": mk.PREC_FP32_DY64, "fp32comp": mk.PREC_FP32_COMP, "fp64": mk.PREC_FP64}[a.precision]
    if a.form == "batch":
        cfg = mk.batch_config(pairs_per_thread=1, substeps_per_launch=0, use_graph=0,
                              max_requests=16, max_nbins=128)
        ctx = mk.Context(0, arena_bytes=mk.batch_workspace_bytes(cfg))
        # N_l of the benchmark's pilot at tol 1e-3, scaled by 1/8
        fixed = [[44000, 22700],
                 [1125000, 380000, 320000, 393000, 318000, 250000, 198000, 169000, 100000],
                 [785000, 100, 100, 100, 100, 100, 100, 100, 100, 100, 2290, 2430, 2600]]
        fixed = [[max(1, x << a.scale) for x in n] for n in fixed]
        probs = [mk.make_problem(precision=prec, n_fixed=n, request=i, **dict(W.periodic_problem(e)))
                 for i, (e, n) in enumerate(zip(W.PERIODIC_EPS, fixed))]
        rs = ctx.estimate_batch(probs, cfg)
        for e, r in zip(W.PERIODIC_EPS, rs):
            print("eps=%g events=%d" % (e, sum(lv["events_f"] + lv["events_c"] for lv in r.levels)))
        ctx.close()
        return
    ctx = mk.Context(0)
    for eps, level, n in ((0.1, 8, 1 << 20), (1e-3, 6, 1 << 20), (0.1, 0, 1 << 22)):
        p = mk.make_problem(precision=prec, **W.periodic_problem(eps))
        st = ctx.run_level(p, level, 0, n << a.scale)
        print("eps=%g level=%d pairs=%d events_f=%d events_c=%d" %
              (eps, level, n << a.scale, st["events_f"], st["events_c"]))
    ctx.close()


if __name__ == "__main__":
    main()
