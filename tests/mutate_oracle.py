"""Mutation check of the oracle's pins (CPU only; not collected by pytest).

Plants one small mistake at a time in a copy of oracle/mlkd_oracle.c: a flipped
sign, a swapped operator, an off-by-one bound, a changed constant, a strict
comparison made non-strict.  It then runs the CPU pin tests against that copy.
A mutant is killed when a test fails or the copy crashes. A survivor is
either equivalent (the change is unobservable) or a gap in the pins.

    python tests/mutate_oracle.py [--jobs 2] [--first 0] [--count 1000] [--workdir DIR]

The mutants cover the method's arithmetic: the uniform recipes and draws, the
coefficients, the KD step, the mapping and aggregation, the cosine sampler
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
SRC = os.path.join(ROOT, "oracle", "mlkd_oracle.c")
PINS = ["tests/test_oracle_rng.py", "tests/test_oracle_coefficients.py",
        "tests/test_oracle_mapping.py", "tests/test_oracle_statistics.py",
        "tests/test_oracle_charfn.py", "tests/test_level_select.py"]
OPERATORS = [(r" \+ ", " - "), (r" - ", " + "), (r" \* ", " / "), (r"floor\(", "ceil("),
             (r" < ", " <= "), (r" <= ", " < "), (r" > ", " >= "), (r" >= ", " > "),
             (r"2\.0", "3.0"), (r"\+ 1\b", "+ 2"), (r"- 1\b", "- 2"), (r"\bexp\(-", "exp("),
             (r"\+= ", "-= "), (r"sqrt\(", "fabs(")]


def mutants(lines):
    """(line index, start, end, replacement) of every operator site in the
    method's arithmetic, in source order."""
    first = next(i for i, l in enumerate(lines) if "orc_u24(uint32_t w)" in l)
    last = next(i for i, l in enumerate(lines) if "ORC_EXPORT int orc_pairs(" in l)
    out = []
    for i in range(first, last):
        s = lines[i].strip()
        if not s or s.startswith(("/*", "*", "//")):
            continue
        code = lines[i].split("/*")[0]
        for pat, rep in OPERATORS:
            for m in re.finditer(pat, code):
                out.append((i, m.start(), m.end(), rep))
    return out


def run_one(lines, mut, workdir):
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
    with open(os.path.join(d, "oracle", "mlkd_oracle.c"), "w") as f:
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
    ap.add_argument("--jobs", type=int, default=2)
    ap.add_argument("--first", type=int, default=0)
    ap.add_argument("--count", type=int, default=1000)
    ap.add_argument("--workdir", default=os.path.join(ROOT, ".mutants"))
    a = ap.parse_args()
    with open(SRC) as f:
        lines = f.read().split("\n")
    ms = mutants(lines)[a.first:a.first + a.count]
    os.makedirs(a.workdir, exist_ok=True)
    work = tempfile.mkdtemp(prefix="mutate_oracle_", dir=a.workdir)
    try:
        with ThreadPoolExecutor(a.jobs) as ex:
            results = list(ex.map(lambda m: run_one(lines, m, work), ms))
    finally:
        shutil.rmtree(work, ignore_errors=True)
    for r in results:
        if not r["killed"]:
            print("SURVIVED line %d: %s  ->  %s" % (r["line"], r["before"], r["after"]))
    killed = sum(r["killed"] for r in results)
    print(json.dumps({"mutants": len(results), "killed": killed, "survived": len(results) - killed}))


if __name__ == "__main__":
    main()
