"""Build the CPU oracle shared library (test infrastructure only).

The whole file is compiled without floating-point contraction so that its
float instantiation is the strict-FP32 reference (no FMA, no fast-math, no
excess precision) on both x86-64 and aarch64 (where GCC contracts by default).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tpcfit_oracle.cpp")
LIB = os.path.join(HERE, "libtpcfit_oracle.so")

FLAGS = ["-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
         "-fexcess-precision=standard", "-fno-finite-math-only", "-frounding-math"]


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["g++", *FLAGS, SRC, "-o", LIB + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
