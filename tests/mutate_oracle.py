"""Mutation check of the oracle's pins (CPU only; not collected by pytest).

Plants one small mistake at a time in a copy of the oracle: a flipped sign, a
swapped operator, an off-by-one bound, a changed constant, a strict comparison
made non-strict.  --target c mutates oracle/mlkd_oracle.c; --target py mutates
the numpy part in oracle/__init__.py (QoIs, bins, level sums, variances, the
sample-count rule, the controller loop, level selection).  It then runs the CPU pin tests against that copy.
A mutant is killed when a test fails or the copy crashes. A survivor is
either equivalent (the change is unobservable) or a gap in the pins.

    python tests/mutate_oracle.py [--target c|py] [--jobs 2] [--first 0] [--count 1000]
                                  [--workdir DIR]

In C the mutants cover the method's arithmetic: the uniform recipes and draws,
the coefficients, the KD step, the mapping and aggregation, the cosine sampler
and the pair driver.  Philox itself is pinned by its published test vectors.
The copies live under --workdir (default: .mutants/ in the repository, which
git ignores) and are removed afterwards.  The library and its header are
linked in, because the level-selection tests call the library's host code.
"""
import argparse
import json
import os
import re
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOURCES = {"c": os.path.join(ROOT, "oracle", "mlkd_oracle.c"),
           "py": os.path.join(ROOT, "oracle", "__init__.py")}
REGIONS = {"c": ("orc_u24(uint32_t w)", "ORC_EXPORT int orc_pairs("),
           "py": ("def qoi_values(", None)}
COMMENT = {"c": ("/*", "*", "//"), "py": ("#", '"""', "'")}
PINS = ["tests/test_oracle_rng.py", "tests/test_oracle_coefficients.py",
        "tests/test_oracle_mapping.py", "tests/test_oracle_statistics.py",
        "tests/test_oracle_charfn.py", "tests/test_level_select.py"]
OPERATORS = [(r" \+ ", " - "), (r" - ", " + "), (r" \* ", " / "), (r"floor\(", "ceil("),
             (r" < ", " <= "), (r" <= ", " < "), (r" > ", " >= "), (r" >= ", " > "),
             (r"2\.0", "3.0"), (r"\+ 1\b", "+ 2"), (r"- 1\b", "- 2"), (r"\bexp\(-", "exp("),
             (r"\+= ", "-= "), (r"sqrt\(", "fabs("), (r"\bmax\(", "min("),
             (r"math\.ceil\(", "math.floor("), (r" == ", " != ")]


def mutants(lines, target="c"):
    """(line index, start, end, replacement) of every operator site in the
    method's arithmetic, in source order."""
    start, stop = REGIONS[target]
    first = next(i for i, l in enumerate(lines) if start in l)
    last = next(i for i, l in enumerate(lines) if stop in l) if stop else len(lines)
    out = []
    in_doc = False
    for i in range(first, last):
        s = lines[i].strip()
        if target == "py" and s.count('"""') == 1:
            in_doc = not in_doc
            continue
        if in_doc or not s or s.startswith(COMMENT[target]):
            continue
        code = lines[i].split("/*" if target == "c" else "#")[0]
        for pat, rep in OPERATORS:
            for m in re.finditer(pat, code):
                out.append((i, m.start(), m.end(), rep))
    return out


def run_one(lines, mut, workdir, target):
    i, a, b, rep = mut
    d = tempfile.mkdtemp(dir=workdir)
    for sub in ("oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copy(os.path.join(ROOT, "workloads.py"), d)
    for sub in ("include", "paper_2004_04071_gb300"):
        os.symlink(os.path.join(ROOT, sub), os.path.join(d, sub))
    changed = list(lines)
    changed[i] = changed[i][:a] + rep + changed[i][b:]
    with open(os.path.join(d, "oracle", os.path.basename(SOURCES[target])), "w") as f:
        f.write("\n".join(changed))
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + PINS,
                           cwd=d, capture_output=True, text=True, timeout=600)
        rc = r.returncode
        failed = [l for l in r.stdout.splitlines() if l.startswith(("FAILED", "ERROR"))]
    except subprocess.TimeoutExpired:
        rc, failed = -9, ["timeout"]
    finally:
        for sub in ("include", "paper_2004_04071_gb300"):
            os.unlink(os.path.join(d, sub))
        shutil.rmtree(d)
    return {"line": i + 1, "before": lines[i].strip(), "after": changed[i].strip(),
            "killed": rc != 0, "by": failed[0] if failed else ("exit %d" % rc if rc else "")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--target", default="c", choices=["c", "py"])
    ap.add_argument("--jobs", type=int, default=2)
    ap.add_argument("--first", type=int, default=0)
    ap.add_argument("--count", type=int, default=1000)
    ap.add_argument("--workdir", default=os.path.join(ROOT, ".mutants"))
    a = ap.parse_args()
    with open(SOURCES[a.target]) as f:
        lines = f.read().split("\n")
    ms = mutants(lines, a.target)[a.first:a.first + a.count]
    os.makedirs(a.workdir, exist_ok=True)
    work = tempfile.mkdtemp(prefix="mutate_oracle_", dir=a.workdir)
    try:
        with ThreadPoolExecutor(a.jobs) as ex:
            results = list(ex.map(lambda m: run_one(lines, m, work, a.target), ms))
    finally:
        shutil.rmtree(work, ignore_errors=True)
    for r in results:
        if not r["killed"]:
            print("SURVIVED line %d: %s  ->  %s" % (r["line"], r["before"], r["after"]))
    killed = sum(r["killed"] for r in results)
    print(json.dumps({"mutants": len(results), "killed": killed, "survived": len(results) - killed}))


if __name__ == "__main__":
    main()
