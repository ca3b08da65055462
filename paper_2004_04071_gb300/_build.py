"""Builds libmlkd.so (the CUDA kernels and the C ABI of include/mlkd.h) in-tree
with nvcc for sm_103a, and libmlkd_checked.so, the same sources with the
device checks of MLKD_CHECKS compiled in (a debug build: a failed bounds check
is recorded and reported as MLKD_EINTERNAL instead of touching memory out of
bounds).  All translation units of both libraries compile in parallel."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libmlkd.so")
LIB_CHECKED = os.path.join(OUT, "libmlkd_checked.so")
SOURCES = ["mlkd_kernels.cu", "mlkd_capi.cu", "mlkd_batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-Xptxas", "-v"]
VARIANTS = {LIB: ("obj", []), LIB_CHECKED: ("obj_checked", ["-DMLKD_CHECKS"])}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "mlkd.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    for lib in VARIANTS:
        if not os.path.exists(lib):
            return False
        t = os.path.getmtime(lib)
        if not all(os.path.getmtime(f) <= t for f in _inputs()):
            return False
    return True


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    cc = nvcc()
    for sub, _ in VARIANTS.values():
        os.makedirs(os.path.join(OUT, sub), exist_ok=True)

    def compile_one(job):
        sub, defs, src = job
        obj = os.path.join(OUT, sub, src + ".o")
        cmd = [cc, *ARCH, *FLAGS, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s %s:\n%s\n%s" % (src, defs, r.stdout, r.stderr))
        return obj, r.stderr

    jobs = [(sub, defs, src) for sub, defs in VARIANTS.values() for src in SOURCES]
    with ThreadPoolExecutor(len(jobs)) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose:
        for _, log in results[:len(SOURCES)]:
            print(log)
    with open(os.path.join(OUT, "ptxas.log"), "w") as fh:
        for (sub, defs, src), (_, log) in zip(jobs, results):
            fh.write("== %s %s ==\n%s\n" % (src, " ".join(defs), log))
    for i, lib in enumerate(VARIANTS):
        objs = [o for o, _ in results[i * len(SOURCES):(i + 1) * len(SOURCES)]]
        tmp = lib + ".tmp%d" % os.getpid()
        r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp] + objs, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
