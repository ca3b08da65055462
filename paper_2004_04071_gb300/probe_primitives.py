"""Builds and runs the primitive-throughput probe (probe_primitives.cu) on
cuda:0 and prints operations per SM per clock for each primitive.

    python -m paper_2004_04071_gb300.probe_primitives

The probe is not part of the library; it measures the FP32, integer and FP64
throughputs that the pair kernel's design is weighed against.
"""
import os
import subprocess
import sys

from paper_2004_04071_gb300 import _build

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "probe_primitives.cu")
EXE = os.path.join(_build.OUT, "probe_primitives")


def build() -> str:
    deps = [SRC, os.path.join(_build.CSRC, "mlkd_device.cuh")]
    if os.path.exists(EXE) and all(os.path.getmtime(d) <= os.path.getmtime(EXE) for d in deps):
        return EXE
    os.makedirs(_build.OUT, exist_ok=True)
    cmd = [_build.nvcc(), *_build.ARCH, "-O3", "-lineinfo", "-std=c++17", SRC, "-o", EXE]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n%s\n%s" % (r.stdout, r.stderr))
    return EXE


def main() -> int:
    exe = build()
    return subprocess.run([exe]).returncode


if __name__ == "__main__":
    sys.exit(main())
