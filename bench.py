"""Throughput of the batched TPC track fit on GB300.

Workload: one time-frame-sized batch of 400,000 synthetic tracks (5% of the
clusters dropped, lengths capped at U{10..152}, sector crossings included),
SoA FP32 clusters and int32 offsets, resident in HBM.  A step is one call of
the library's fit on that batch (length ordering + fast FP32 fit).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank fits its own batch of
the same size (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fitted tracks/s on 1 GB300 (fit, fit+adjoint) vs plain; % of FP32 roofline"
UNIT = "tracks/s"
WORKLOAD = "time-frame batch: 400,000 tracks, 5% clusters dropped, lengths U{10..152}, Bz 0.5 T, 36 sectors x 152 rows"
N_TRACKS = 400_000


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_mhz: float, n_sm: int = 152) -> float:
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic(kernel_key: str):
    """DRAM bytes per launch from a committed ncu summary, if it matches the current sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    ent = t.get(kernel_key)
    if not ent or ent.get("source_sha") != _source_sha():
        return None
    return ent.get("dram_bytes_per_launch")


def _source_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2511_17018_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h", ".cpp")):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(fn.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def cpu_baseline(frame, budget_s: float = 20.0):
    """The FP64 oracle as it stands, on this host's cores, over a bounded sample."""
    import oracle
    threads = oracle.default_threads()
    n = frame.n_tracks
    take = min(n, 50_000)
    sub = frame.subset(np.arange(take))
    t0 = time.perf_counter()
    oracle.fit(sub, "f64", nthreads=threads)
    dt = time.perf_counter() - t0
    reps = 1
    if dt < budget_s / 4:
        # grow the sample up to the whole batch within the budget
        take = int(min(n, take * max(1.0, (budget_s / 2) / max(dt, 1e-3))))
        sub = frame.subset(np.arange(take))
        t0 = time.perf_counter()
        oracle.fit(sub, "f64", nthreads=threads)
        dt = time.perf_counter() - t0
    return {"value": take * reps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {take} tracks of the batch, FP64 oracle, {threads} threads, {dt:.2f} s"}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    from paper_2511_17018_gb300 import synth
    fr = synth.config2(N_TRACKS)
    import oracle
    threads = oracle.default_threads()
    take = min(fr.n_tracks, 100_000)
    sub = fr.subset(np.arange(take))
    for _ in range(args.warmup):
        oracle.fit(sub, "f64", nthreads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fit(sub, "f64", nthreads=threads)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = take * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_tracks_per_step": take},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"first {take} of {fr.n_tracks} tracks per step, FP64 oracle"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def e2e_run(fitter, fr, out, steps, tf, torch):
    """Tracks/s through tpcfit_fit_host with pinned host buffers: every step
    copies the batch to the device, fits and copies the results back."""
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
           (("y", fr.y), ("z", fr.z), ("rowsec", fr.rowsec.view(np.int16)), ("offsets", fr.offsets),
            ("seeds", fr.seeds))}
    hout = {k: torch.empty(tuple(v.shape), dtype=v.dtype).pin_memory() for k, v in out.items()}
    hnp = {k: v.numpy() for k, v in hout.items()}
    args_np = (pin["y"].numpy(), pin["z"].numpy(), pin["rowsec"].numpy().view(np.uint16), pin["offsets"].numpy(),
               pin["seeds"].numpy())
    for _ in range(2):
        tf.tpcfit_fit_host(fitter.h, *args_np, out=hnp)
    n = max(3, min(50, steps // 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n):
        tf.tpcfit_fit_host(fitter.h, *args_np, out=hnp)
    return fr.n_tracks / ((time.perf_counter() - t0) / n)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["fast", "det"], default="fast")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tracks", type=int, default=N_TRACKS,
                    help="batch size override (profiling of smaller cases only; the bench value uses the default)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)

    from paper_2511_17018_gb300 import flops, synth
    from paper_2511_17018_gb300 import tpcfit as tf

    fr = synth.generate(args.tracks, 2 + 1000 * rank, drop_p=0.05, cap_lengths=True)
    lengths = fr.lengths()
    dev = tf.frame_to_device(fr)
    fitter = tf.Fitter(fr.geometry, fr.bz, deterministic=(args.mode == "det"))
    tf.tpcfit_reserve(fitter.h, fr.n_tracks, fr.n_hits)
    out = tf.empty_outputs(fr.n_tracks)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        fitter.fit(dev, out)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            fitter.fit(dev, out)
            ev[i][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = t_start.elapsed_time(t_end)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    st, code, trk = fitter.status()
    if st != 0:
        raise RuntimeError(f"device reported invalid input: code {code} track {trk}")
    ndf = out["ndf"].cpu().numpy()

    # end to end through the host-buffer entry point (pinned host memory)
    h2d = 10 * fr.n_hits + 4 * (fr.n_tracks + 1) + 20 * fr.n_tracks
    d2h = 88 * fr.n_tracks
    e2e = None
    if not args.no_e2e:
        e2e = {"value": e2e_run(fitter, fr, out, args.steps, tf, torch), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank != 0:
        fitter.close()
        if world > 1:
            dist.destroy_process_group()
        return

    peaks, peak_src = _peaks()
    mean_step_s = statistics.mean(step_ms) / 1e3
    alg_flops = flops.fit_flops(lengths)
    peak_tf = fp32_peak_tflops(float(peaks.get("sm_max_mhz", 2070.0)))
    achieved_tf = alg_flops / mean_step_s / 1e12
    value = world * fr.n_tracks * args.steps / (total_ms / 1e3)
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mode": args.mode, "tracks": fr.n_tracks, "hits": fr.n_hits,
                   "mean_hits_per_track": float(lengths.mean()),
                   "l2": "inputs larger than L2 (clusters %.0f MB > 126 MB), no flush" % (10 * fr.n_hits / 1e6),
                   "fitted_fraction": float(np.mean(ndf > 0))},
        "hits_per_s": value * float(lengths.mean()),
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": achieved_tf / peak_tf, "traffic": _traffic("fit_fast" if args.mode == "fast" else "fit_det"),
                     "kernel": "fit_kernel (+ length ordering) per tpcfit_fit call",
                     "algorithmic_flops_per_launch": alg_flops,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                                    f"(sm_max_mhz, {peak_src} peaks file)",
                     "frac_at_sampled_clock": (achieved_tf / fp32_peak_tflops(clocks["sm_mhz"]))
                     if clocks.get("sm_mhz") else None},
        "e2e": e2e,
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(fr)
    fitter.close()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
