"""Build libtpcfit.so in-tree for sm_103a.

One nvcc invocation per translation unit, in parallel, each with the flags of
its module (the per-kernel compilation units of Sec. 3): the fast fit with FMA
contraction and approximate division / square root, the deterministic fit with
-fmad=false and IEEE division / square root.  Only the tpcfit_* C symbols are
exported.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", "tpcfit")
LIB = os.path.join(HERE, "libtpcfit.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", f"-I{INC}", f"-I{CSRC}",
          "--expt-relaxed-constexpr"]
FAST = ["-fmad=true", "-prec-div=false", "-prec-sqrt=false", "-ftz=true"]
DET = ["-fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false"]

UNITS = {
    "tpcfit_host.cpp": [],
    "fit_fast.cu": FAST,
    "fit_det.cu": DET,
    "length_order.cu": [],
    "tpcfit_noalloc.cu": [],
    "key_reduce.cu": [],
}


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _sources():
    return [os.path.join(CSRC, u) for u in UNITS] + [os.path.join(CSRC, f) for f in os.listdir(CSRC)
                                                    if f.endswith((".cuh", ".h", ".map"))] + [
        os.path.join(INC, "tpcfit.h"), os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources() if os.path.exists(s))


def _compile(unit: str, extra, verbose_ptxas: bool):
    src = os.path.join(CSRC, unit)
    obj = os.path.join(BUILD, unit + ".o")
    lang = ["-x", "cu"] if unit.endswith(".cu") else []
    cmd = [nvcc(), *ARCH, *COMMON, *extra, *lang, "-c", src, "-o", obj]
    if verbose_ptxas and unit.endswith(".cu"):
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        futs = [ex.submit(_compile, u, f, verbose_ptxas) for u, f in UNITS.items()]
        results = [f.result() for f in futs]
    if verbose_ptxas:
        for _, log in results:
            if log:
                print(log, file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs,
           "-Xlinker", f"--version-script={os.path.join(CSRC, 'exports.map')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
