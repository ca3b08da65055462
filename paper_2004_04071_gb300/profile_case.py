"""Small, fixed pair-kernel launches for profiling with ncu.

    python -m paper_2004_04071_gb300.profile_case [--precision fp32|fp32comp|fp64]

Runs three launches of the pair kernel on cuda:0, each over 2^20 pairs (2^22
for the level-0 case), on the periodic problem of the benchmark:
  1. eps = 0.1, level 8  (mixed regime, R dt = 0.2)
  2. eps = 1e-3, level 6 (deep diffusive, one event per fine step)
  3. eps = 0.1, level 0  (initialisation-dominated, two events per path)
and prints the event counts.  Device memory held: the 0.7 MB context arena.
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
    a = ap.parse_args()
    prec = {"fp32": mk.PREC_FP32_DY64, "fp32comp": mk.PREC_FP32_COMP, "fp64": mk.PREC_FP64}[a.precision]
    ctx = mk.Context(0)
    for eps, level, n in ((0.1, 8, 1 << 20), (1e-3, 6, 1 << 20), (0.1, 0, 1 << 22)):
        p = mk.make_problem(precision=prec, **W.periodic_problem(eps))
        st = ctx.run_level(p, level, 0, n << a.scale)
        print("eps=%g level=%d pairs=%d events_f=%d events_c=%d" %
              (eps, level, n << a.scale, st["events_f"], st["events_c"]))
    ctx.close()


if __name__ == "__main__":
    main()
