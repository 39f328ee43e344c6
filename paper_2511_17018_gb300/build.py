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
    "rtc.cpp": [],
    "fit_fast.cu": FAST,
    "fit_det.cu": DET,
    "length_order.cu": [],
    "tpcfit_noalloc.cu": [],
    "key_reduce.cu": [],
    "fp32_peak.cu": [],
    "reject.cu": [],
}


# Device sources the library carries for run-time compilation (Sec. 5).
RTC_SOURCES = ("kernel_abi.h", "device_util.cuh", "fit_core.cuh", "ud_filter.cuh")
RTC_EMBED = os.path.join(BUILD, "rtc_sources.cpp")


def write_rtc_embed() -> str:
    """The device sources as string constants (kRtcSources), for NVRTC."""
    delim = "TPCFIT_SRC"
    parts = ["// Generated by build.py: device sources embedded for run-time compilation.",
             "namespace tpcfit {", f"extern const int kRtcSourceCount = {len(RTC_SOURCES)};",
             "extern const char* const kRtcSourceNames[] = {" + ", ".join(f'"{n}"' for n in RTC_SOURCES) + "};",
             "extern const char* const kRtcSources[] = {"]
    for n in RTC_SOURCES:
        with open(os.path.join(CSRC, n)) as f:
            text = f.read()
        assert f"){delim}\"" not in text
        parts.append(f'R"{delim}({text}){delim}",')
    parts += ["};", "}  // namespace tpcfit", ""]
    body = "\n".join(parts)
    if not os.path.exists(RTC_EMBED) or open(RTC_EMBED).read() != body:
        with open(RTC_EMBED, "w") as f:
            f.write(body)
    return RTC_EMBED


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
    src = unit if os.path.isabs(unit) else os.path.join(CSRC, unit)
    obj = os.path.join(BUILD, os.path.basename(unit) + ".o")
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
    units = dict(UNITS)
    units[write_rtc_embed()] = []
    with cf.ThreadPoolExecutor(max_workers=len(units)) as ex:
        futs = [ex.submit(_compile, u, f, verbose_ptxas) for u, f in units.items()]
        results = [f.result() for f in futs]
    if verbose_ptxas:
        for _, log in results:
            if log:
                print(log, file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs,
           "-Xlinker", f"--version-script={os.path.join(CSRC, 'exports.map')}", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
