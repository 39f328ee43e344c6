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
import gc
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
    """Hash of the kernel sources (.cu, .cuh and the headers they include); the
    host-side .cpp files do not change what a kernel reads and writes."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2511_17018_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(fn.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def _oracle_fit_adjoint(sub, threads):
    """The oracle's fit with its FP64 forward-mode gradient of sum(chi2) / N."""
    import oracle
    w = np.full(sub.n_tracks, 1.0 / max(sub.n_tracks, 1))
    return oracle.grad(sub, weights=w, nthreads=threads)


def cpu_baseline(frame, budget_s: float = 15.0):
    """The oracle as it stands on this host's cores, on a bounded sample of the
    batch: fit + gradient (the metric's step) and, for context, the plain fit."""
    import oracle
    threads = oracle.default_threads()
    probe = frame.subset(np.arange(min(frame.n_tracks, 256)))
    t0 = time.perf_counter()
    _oracle_fit_adjoint(probe, threads)
    per_track = (time.perf_counter() - t0) / probe.n_tracks
    take = int(min(frame.n_tracks, max(256, budget_s / max(per_track, 1e-9))))
    sub = frame.subset(np.arange(take))
    t0 = time.perf_counter()
    _oracle_fit_adjoint(sub, threads)
    dt = time.perf_counter() - t0
    plain_take = min(frame.n_tracks, 100_000)
    psub = frame.subset(np.arange(plain_take))
    t1 = time.perf_counter()
    oracle.fit(psub, "f64", nthreads=threads)
    pdt = time.perf_counter() - t1
    # the same two legs on one thread, on smaller samples (about 3 s in all)
    one = frame.subset(np.arange(min(frame.n_tracks, 256)))
    t2 = time.perf_counter()
    _oracle_fit_adjoint(one, 1)
    odt = time.perf_counter() - t2
    one_plain = frame.subset(np.arange(min(frame.n_tracks, 20_000)))
    t3 = time.perf_counter()
    oracle.fit(one_plain, "f64", nthreads=1)
    opdt = time.perf_counter() - t3
    return {"value": take / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {take} tracks of the batch: FP64 fit + forward-mode gradient, {threads} threads, "
                      f"{dt:.1f} s",
            "plain_fit": {"value": plain_take / pdt, "unit": UNIT,
                          "sample": f"first {plain_take} tracks, FP64 fit only, {pdt:.2f} s"},
            "one_thread": {"value": one.n_tracks / odt, "plain_fit": one_plain.n_tracks / opdt, "unit": UNIT,
                           "sample": f"first {one.n_tracks} tracks (fit + gradient, {odt:.2f} s) and first "
                                     f"{one_plain.n_tracks} tracks (FP64 fit only, {opdt:.2f} s), 1 thread"}}


def run_reference(args, rank: int, world: int):
    """The oracle on the host cores, timed on this bench's workload and metric
    (fit + gradient per track); each step is a bounded sample sized so that the
    whole run takes about two minutes."""
    if rank != 0:
        return
    from paper_2511_17018_gb300 import synth
    import oracle
    fr = synth.time_frame(N_TRACKS)
    threads = oracle.default_threads()
    probe = fr.subset(np.arange(256))
    t0 = time.perf_counter()
    _oracle_fit_adjoint(probe, threads)
    per_track = (time.perf_counter() - t0) / 256
    budget = 120.0 / max(1, args.steps + args.warmup)
    take = int(min(fr.n_tracks, max(64, budget / max(per_track, 1e-9))))
    sub = fr.subset(np.arange(take))
    for _ in range(args.warmup):
        _oracle_fit_adjoint(sub, threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _oracle_fit_adjoint(sub, threads)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = take * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": "FP64 fit + forward-mode gradient of the mean chi2",
                   "sample_tracks_per_step": take},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"first {take} of {fr.n_tracks} tracks per step, FP64 fit + gradient"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_fp32_peak(tf, torch, device_index: int, seconds: float = 1.5) -> dict:
    """The FP32 peak of this GPU from the library's FMA-chain microbenchmark
    (scalar FMAs and paired fma.f32x2, each one launch of about `seconds`,
    clocks sampled during it); the larger of the two is the roofline's
    denominator.  Cross-check: SMs x 128 FP32 lanes x 2 x the sampled clock."""
    res = {}
    for mode, name in ((0, "ffma"), (1, "ffma2")):
        fl, ms = tf.tpcfit_fp32_peak(mode, 2000)           # calibration launch
        iters = max(2000, int(2000 * seconds * 1e3 / max(ms, 1e-3)))
        torch.cuda.synchronize()
        with ClockSampler(device_index) as clk:
            fl, ms = tf.tpcfit_fp32_peak(mode, iters)
        res[name] = {"tflops": fl / (ms / 1e3) / 1e12, "ms": ms, "clocks": clk.summary()}
    best = max(res.values(), key=lambda r: r["tflops"])
    sms = torch.cuda.get_device_properties(device_index).multi_processor_count
    mhz = best["clocks"].get("sm_mhz")
    return {"tflops": best["tflops"], "ffma": res["ffma"], "ffma2": res["ffma2"], "sms": sms,
            "nominal_at_sampled_clock_tflops": fp32_peak_tflops(mhz, sms) if mhz else None}


def rank_seed(rank: int) -> int:
    """Each rank fits its own batch of the same size (weak scaling)."""
    return 2 + 1000 * rank


def combine_ranks(dist, torch, device, step_ms: float, rates: list) -> tuple:
    """Whole-job view of per-rank numbers: the slowest rank's step time (MAX)
    and, for per-rank throughputs, world size x the slowest rank (MIN)."""
    world = dist.get_world_size()
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    r = torch.tensor(rates if rates else [0.0], dtype=torch.float64, device=device)
    dist.all_reduce(r, op=dist.ReduceOp.MIN)
    return float(t.item()), [float(v) * world for v in r.tolist()][: len(rates)]


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
    n = max(10, min(50, steps // 4))
    torch.cuda.synchronize()
    with _NoGC():
        t0 = time.perf_counter()
        for _ in range(n):
            tf.tpcfit_fit_host(fitter.h, *args_np, out=hnp)
        dt = time.perf_counter() - t0
    return fr.n_tracks / (dt / n)


class _NoGC:
    """The timed host loops run with Python's garbage collector paused (as
    timeit does): a collection pass over the objects the bench holds by then
    costs milliseconds, which a 0.2 s loop would otherwise count as the
    library's time."""

    def __enter__(self):
        self.was = gc.isenabled()
        gc.disable()
        return self

    def __exit__(self, *a):
        if self.was:
            gc.enable()


def _e2e_host_buffers(fr, torch):
    """The batch and dL/dchi2 in pinned host memory, and two sets of pinned
    host outputs (numpy views)."""
    n = fr.n_tracks
    pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
           (fr.y, fr.z, fr.rowsec.view(np.int16), fr.offsets, fr.seeds, np.full(n, 1.0 / n, np.float32))]
    y, z, rs, off, sd, g = (t.numpy() for t in pin)
    args = (y, z, rs.view(np.uint16), off, sd, g)

    def outputs():
        t = {"chi2": torch.empty(n).pin_memory(), "ndf": torch.empty(n, dtype=torch.int32).pin_memory(),
             "grad_align": torch.empty((36, 152, 2)).pin_memory(), "grad_seeds": torch.empty((5, n)).pin_memory()}
        return t, {k: v.numpy() for k, v in t.items()}
    outs = [outputs() for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for t in pin)
    d2h = sum(v.numel() * v.element_size() for v in outs[0][0].values())
    return pin, args, outs, h2d, d2h


def e2e_fit_adjoint(fitter, fr, steps, tf, torch):
    """Tracks/s of fit + adjoint through the C-ABI host-buffer call
    (tpcfit_fit_adjoint_host): each step copies the batch and dL/dchi2 from
    pinned host memory, fits with checkpoints, runs the adjoint and copies chi2,
    ndf and both gradients back; the host waits for each step before the next."""
    _pin, args, outs, h2d, d2h = _e2e_host_buffers(fr, torch)
    stream = torch.cuda.current_stream()

    def step():
        tf.tpcfit_fit_adjoint_host(fitter.h, *args, out=outs[0][1])
        stream.synchronize()

    for _ in range(2):
        step()
    m = max(10, min(50, steps // 4))
    with _NoGC():
        t0 = time.perf_counter()
        for _ in range(m):
            step()
        dt = (time.perf_counter() - t0) / m
    return fr.n_tracks / dt, h2d, d2h


def e2e_fit_adjoint_pipelined(fitter, fr, steps, tf, torch):
    """The same calls issued back to back: the library copies a call's inputs
    on its own copy stream into one of two staging sets, so step k+1's copies
    overlap step k's fit and adjoint; the host waits for every step's results
    (step k-1's while step k runs) before reusing their buffers."""
    _pin, args, outs, h2d, d2h = _e2e_host_buffers(fr, torch)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event() for _ in range(2)]

    def run(m):
        for j in range(m):
            if j >= 2:
                ev[j % 2].synchronize()  # step j - 2's results were read before the buffers are reused
            tf.tpcfit_fit_adjoint_host(fitter.h, *args, out=outs[j % 2][1])
            ev[j % 2].record(stream)
            if j >= 1:
                ev[(j - 1) % 2].synchronize()  # the host has step j - 1's results
        ev[(m - 1) % 2].synchronize()

    run(3)
    m = max(10, min(50, steps // 4))
    with _NoGC():
        t0 = time.perf_counter()
        run(m)
        dt = (time.perf_counter() - t0) / m
    return fr.n_tracks / dt, h2d, d2h


def run_batched_frames(args, tf, torch, synth, flops, peak_tf):
    """256 frames, track counts log-uniform on [1e3, 2e5] (8.99M tracks), one
    persistent launch replayed from a CUDA graph; launch shape from the autotuner."""
    from paper_2511_17018_gb300 import autotune
    from paper_2511_17018_gb300.frames import FrameBatch, GraphedFrameFit, fit_frames
    pool, picks = synth.batched_frames(pool_tracks=args.pool_tracks)
    batch = FrameBatch.from_pool(pool, picks)
    lengths = np.diff(batch.offsets.cpu().numpy().astype(np.int64))
    res = {"workload": "256 frames, tracks per frame log-uniform on [1e3, 2e5], drawn (seeded, with replacement) "
                       f"from a simulated pool of {pool.n_tracks} tracks (5% drop, lengths U{{10..152}}): frames "
                       "repeat pool tracks, so they are not independent simulations",
           "frames": batch.n_frames, "tracks": batch.n_tracks, "hits": batch.n_hits}
    for mode in ("fast", "det"):
        f = tf.Fitter(pool.geometry, pool.bz, deterministic=(mode == "det"))
        tf.tpcfit_reserve(f.h, batch.n_tracks, batch.n_hits)
        out = tf.empty_outputs(batch.n_tracks)
        best = autotune.tune(f, batch.dev(), lengths, mode=mode, reps=2, cache_path=None,
                             fit_call=lambda: fit_frames(f, batch, out))
        del out
        g = GraphedFrameFit(f, batch)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        s.record()
        for _ in range(reps):
            g.replay()
        e.record()
        torch.cuda.synchronize()
        ms = s.elapsed_time(e) / reps
        # the U-D fit in fast mode with one lane per track, else the square-root form
        form = 1 if (mode == "fast" and best["lanes_per_track"] == 1) else 0
        tfl = flops.fit_flops(lengths, form) / (ms / 1e3) / 1e12
        tfm = flops.method_fit_flops(lengths) / (ms / 1e3) / 1e12
        res[mode] = {"tracks_per_s": batch.n_tracks / (ms / 1e3), "ms_per_batch": ms,
                     "hits_per_s": batch.n_hits / (ms / 1e3), "frac_method": tfm / peak_tf, "frac_impl": tfl / peak_tf,
                     "config": {k: best[k] for k in ("lanes_per_track", "rows_per_stage", "warps_per_block",
                                                     "sort_by_length")},
                     "sweep_by_lanes_ms": {k: round(v["ms"], 3) for k, v in best["by_lanes"].items()},
                     "fitted_fraction": float((g.out["ndf"] > 0).float().mean().item())}
        del g
        f.close()
    if not args.no_cpu_baseline:
        # the oracle's FP64 fit on a slice of the pool the frames are drawn
        # from, its per-track rate extrapolated to the batch
        import oracle
        threads = oracle.default_threads()
        take = min(pool.n_tracks, 100_000)
        sub = pool.subset(np.arange(take))
        t0 = time.perf_counter()
        oracle.fit(sub, "f64", nthreads=threads)
        dt = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": take / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": f"first {take} tracks of the frames' pool: FP64 fit, {threads} threads, "
                                         f"{dt:.2f} s",
                               "extrapolated_batch_s": batch.n_tracks / (take / dt),
                               "note": "the sample's per-track rate extrapolated to the batch's tracks"}
    del batch
    torch.cuda.empty_cache()
    return res


def run_alignment_loop(args, tf, torch, synth):
    """2,000,000 tracks with injected offsets N(0, 0.05 cm); 50 iterations of
    fit + adjoint + Adam on the device (CUDA graph)."""
    from paper_2511_17018_gb300 import align
    d_true = synth.alignment_offsets(5)
    fr = synth.generate(args.align_tracks, 5, drop_p=0.05, cap_lengths=True, d_true=d_true)
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz)
    loop = align.AlignmentLoop(f, dev, lr=5e-3)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    losses = loop.run(args.align_iters)
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / args.align_iters
    raw0, proj0 = align.recovery(np.zeros_like(d_true), d_true, fr.geometry.row_x)
    raw, proj = align.recovery(loop.d.cpu().numpy(), d_true, fr.geometry.row_x)
    f.close()
    return {"workload": f"{fr.n_tracks} tracks, injected offsets N(0, 0.05 cm), {args.align_iters} iterations, "
                        "Adam lr 5e-3", "tracks_per_s_per_iteration": fr.n_tracks / (ms / 1e3), "ms_per_iteration": ms,
            "loss_first_last": [float(losses[0]), float(losses[-1])],
            "rms_cm_initial": {"raw": raw0, "weak_modes_removed": proj0},
            "rms_cm_final": {"raw": raw, "weak_modes_removed": proj}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["fast", "det"], default="fast")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched-frames and alignment-loop workloads")
    ap.add_argument("--pool-tracks", type=int, default=1_000_000)
    ap.add_argument("--align-tracks", type=int, default=2_000_000)
    ap.add_argument("--align-iters", type=int, default=50)
    ap.add_argument("--tracks", type=int, default=N_TRACKS,
                    help="batch size override (profiling of smaller cases only; the bench value uses the default)")
    ap.add_argument("--bwd-warps", type=int, default=None, help="adjoint warps per block (library default if unset)")
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

    fr = synth.generate(args.tracks, rank_seed(rank), drop_p=0.05, cap_lengths=True)
    lengths = fr.lengths()
    dev = tf.frame_to_device(fr)
    fitter = tf.Fitter(fr.geometry, fr.bz, deterministic=(args.mode == "det"))
    if args.bwd_warps is not None:
        fitter.set_backward_config(args.bwd_warps)
    tf.tpcfit_reserve(fitter.h, fr.n_tracks, fr.n_hits)
    out = tf.empty_outputs(fr.n_tracks)
    g_chi2 = torch.full((fr.n_tracks,), 1.0 / fr.n_tracks, dtype=torch.float32, device="cuda")
    g_align = torch.empty(36 * 152 * 2, dtype=torch.float32, device="cuda")
    g_seeds = torch.empty((5, fr.n_tracks), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def fit_adjoint():
        fitter.fit(dev, out)
        tf.tpcfit_fit_backward(fitter.h, dev["y"], dev["z"], dev["rowsec"], dev["offsets"], out["ndf"], g_chi2,
                               g_align, g_seeds)

    def timed(fn, steps, split=False):
        """device time of `steps` calls (CUDA events on the launching stream)."""
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(steps):
            ev[i][0].record(stream)
            fn(ev[i][1])
            ev[i][2].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        per = [(a.elapsed_time(b), b.elapsed_time(c)) for a, b, c in ev]
        return t0.elapsed_time(t1), per

    def step_fa(mid):
        fitter.fit(dev, out)
        mid.record(stream)
        tf.tpcfit_fit_backward(fitter.h, dev["y"], dev["z"], dev["rowsec"], dev["offsets"], out["ndf"], g_chi2,
                               g_align, g_seeds)

    def step_fit(mid):
        fitter.fit(dev, out)
        mid.record(stream)

    # ---- the step: fit with checkpoints + adjoint
    fitter.set_record(True)
    for _ in range(args.warmup):
        fit_adjoint()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        total_ms, per = timed(step_fa, args.steps)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if world > 1:
        total_ms, _ = combine_ranks(dist, torch, "cuda", total_ms, [])
    st, code, trk = fitter.status()
    if st != 0:
        raise RuntimeError(f"device reported invalid input: code {code} track {trk}")
    ndf = out["ndf"].cpu().numpy()
    fit_rec_ms = statistics.mean(p[0] for p in per)
    bwd_ms = statistics.mean(p[1] for p in per)

    # ---- end to end through the public API with host buffers, on the same
    # handle right after the device-timed step
    h2d = 10 * fr.n_hits + 4 * (fr.n_tracks + 1) + 20 * fr.n_tracks
    d2h = 88 * fr.n_tracks
    e2e = e2e_plain = None
    if not args.no_e2e:
        fitter.set_record(False)
        e2e_plain = {"value": e2e_run(fitter, fr, out, args.steps, tf, torch), "unit": UNIT,
                     "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        fitter.set_record(True)
        v_serial, _, _ = e2e_fit_adjoint(fitter, fr, args.steps, tf, torch)
        v, hb, db = e2e_fit_adjoint_pipelined(fitter, fr, args.steps, tf, torch)
        if world > 1:  # whole job: every rank streams its own batch; the slowest rank sets the pace
            _, (v, e2e_plain["value"], v_serial) = combine_ranks(dist, torch, "cuda", 0.0,
                                                                 [v, e2e_plain["value"], v_serial])
        e2e = {"value": v, "unit": UNIT, "h2d_bytes_per_step": hb, "d2h_bytes_per_step": db,
               "call": "tpcfit_fit_adjoint_host (C ABI, pinned host buffers), one call per step",
               "pipelining": "calls issued back to back: step k+1's host-to-device copies (library copy stream, "
                             "second staging set) overlap step k's fit and adjoint; the host waits for every "
                             "step's results",
               "serial_value": v_serial}

    # the smoother below reads the recording of the device-buffer fit
    fitter.set_record(True)
    fitter.fit(dev, out)
    torch.cuda.synchronize()

    # ---- the two-filter smoother of the recorded fit (per-cluster outlier test)
    sm = dict(resid=torch.empty((fr.n_hits, 2), device="cuda"), rcov=torch.empty((fr.n_hits, 3), device="cuda"),
              chi2=torch.empty(fr.n_hits, device="cuda"))

    def step_smooth(mid):
        tf.tpcfit_smooth(fitter.h, dev["y"], dev["z"], dev["rowsec"], dev["offsets"], out["ndf"], sm["resid"],
                         sm["rcov"], sm["chi2"])
        mid.record(stream)

    for _ in range(args.warmup):
        step_smooth(torch.cuda.Event())
    torch.cuda.synchronize()
    _, sm_per = timed(step_smooth, max(5, args.steps // 4))
    smooth_ms = statistics.mean(p[0] for p in sm_per)
    # outlier rejection on the smoother's chi2 (2-dof cut 16): kept clusters copied, new offsets
    rj = dict(y=torch.empty(fr.n_hits, device="cuda"), z=torch.empty(fr.n_hits, device="cuda"),
              rs=torch.empty(fr.n_hits, dtype=torch.int16, device="cuda"),
              off=torch.empty(fr.n_tracks + 1, dtype=torch.int32, device="cuda"))

    def step_reject(mid):
        tf.tpcfit_reject_outliers(fitter.h, dev["y"], dev["z"], dev["rowsec"], dev["offsets"], sm["chi2"], 16.0,
                                  rj["y"], rj["z"], rj["rs"], rj["off"])
        mid.record(stream)

    for _ in range(args.warmup):
        step_reject(torch.cuda.Event())
    torch.cuda.synchronize()
    _, rj_per = timed(step_reject, max(5, args.steps // 4))
    reject_ms = statistics.mean(p[0] for p in rj_per)
    reject_kept = int(rj["off"][-1].item())
    del sm, rj
    # the smoothed state and covariance at every cluster
    ss = dict(state=torch.empty((fr.n_hits, 5), device="cuda"), cov=torch.empty((fr.n_hits, 15), device="cuda"))

    def step_states(mid):
        tf.tpcfit_smooth_states(fitter.h, dev["y"], dev["z"], dev["rowsec"], dev["offsets"], out["ndf"],
                                ss["state"], ss["cov"])
        mid.record(stream)

    for _ in range(args.warmup):
        step_states(torch.cuda.Event())
    torch.cuda.synchronize()
    _, ss_per = timed(step_states, max(5, args.steps // 4))
    states_ms = statistics.mean(p[0] for p in ss_per)
    del ss

    # ---- the plain fit (no checkpoints)
    fitter.set_record(False)
    for _ in range(args.warmup):
        fitter.fit(dev, out)
    torch.cuda.synchronize()
    plain_steps = max(args.steps, 20)
    plain_total, plain_per = timed(step_fit, plain_steps)
    plain_ms = statistics.mean(p[0] for p in plain_per)

    # ---- the same plain fit with the kernel compiled at run time for this
    # frame's constants (Sec. 5); the first call compiles and loads it
    rtc = None
    if tf.tpcfit_rtc_available():
        fitter.set_rtc(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fitter.fit(dev, out)
        torch.cuda.synchronize()
        first_s = time.perf_counter() - t0
        for _ in range(args.warmup):
            fitter.fit(dev, out)
        torch.cuda.synchronize()
        _, rtc_per = timed(step_fit, plain_steps)
        rtc = {"ms": statistics.mean(p[0] for p in rtc_per), "first_call_s": first_s}
        fitter.set_rtc(False)

    # ---- the same plain fit with the material layers of the TPC gas at every row
    from paper_2511_17018_gb300 import synth as _synth
    fitter.set_material(_synth.TPC_GAS)
    for _ in range(args.warmup):
        fitter.fit(dev, out)
    torch.cuda.synchronize()
    _, mat_per = timed(step_fit, plain_steps)
    mat_ms = statistics.mean(p[0] for p in mat_per)
    # and the fit + adjoint step through the layers
    fitter.set_record(True)
    for _ in range(args.warmup):
        step_fa(torch.cuda.Event())
    torch.cuda.synchronize()
    _, mat_fa_per = timed(step_fa, max(5, args.steps // 4))
    fitter.set_record(False)
    fitter.set_material(None)

    # ---- the same plain fit in the field map Bz (1 + 0.3 (r/250)^2 - 0.2 (z/250)^2)
    fitter.set_field(_synth.FieldMap(0.3, -0.2))
    for _ in range(args.warmup):
        fitter.fit(dev, out)
    torch.cuda.synchronize()
    _, fld_per = timed(step_fit, plain_steps)
    fld_ms = statistics.mean(p[0] for p in fld_per)
    fitter.set_record(True)
    for _ in range(args.warmup):
        step_fa(torch.cuda.Event())
    torch.cuda.synchronize()
    _, fld_fa_per = timed(step_fa, max(5, args.steps // 4))
    fitter.set_record(False)
    fitter.set_field(None)

    # ---- deterministic mode on the same frame: plain fit and fit + adjoint
    det = None
    if args.mode == "fast":
        fitter.set_mode(True)
        fitter.set_record(False)
        for _ in range(args.warmup):
            fitter.fit(dev, out)
        torch.cuda.synchronize()
        _, det_fit_per = timed(step_fit, max(10, args.steps // 4))
        fitter.set_record(True)
        for _ in range(args.warmup):
            fit_adjoint()
        torch.cuda.synchronize()
        _, det_fa_per = timed(step_fa, max(10, args.steps // 4))
        fitter.set_record(False)
        fitter.set_mode(False)
        det = {"plain_fit_ms": statistics.mean(p[0] for p in det_fit_per),
               "fit_ms": statistics.mean(p[0] for p in det_fa_per),
               "backward_ms": statistics.mean(p[1] for p in det_fa_per)}

    # ---- the square-root factor (Potter's updates) in place of U-D in fast mode
    sqrt_form = None
    if args.mode == "fast":
        fitter.set_fit_form(0)
        fitter.set_backward_form(0)
        fitter.set_record(False)
        for _ in range(args.warmup):
            fitter.fit(dev, out)
        torch.cuda.synchronize()
        _, sq_fit_per = timed(step_fit, max(10, args.steps // 4))
        fitter.set_record(True)
        for _ in range(args.warmup):
            fit_adjoint()
        torch.cuda.synchronize()
        _, sq_fa_per = timed(step_fa, max(10, args.steps // 4))
        fitter.set_record(False)
        fitter.set_fit_form(1)
        fitter.set_backward_form(1)
        sqrt_form = {"plain_fit_ms": statistics.mean(p[0] for p in sq_fit_per),
                     "fit_ms": statistics.mean(p[0] for p in sq_fa_per),
                     "backward_ms": statistics.mean(p[1] for p in sq_fa_per)}

    if rank != 0:
        fitter.close()
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- the FP32 peak of this GPU, measured (the roofline's denominator)
    peak = measure_fp32_peak(tf, torch, local)
    peak_tf = peak["tflops"]
    value = world * fr.n_tracks * args.steps / (total_ms / 1e3)
    clocks = clk.summary()
    step_ms = total_ms / args.steps
    mhits = float(lengths.mean())

    def frac2(impl_flops, method_flops, ms):
        """achieved TFLOP/s and fraction of the measured peak on both counts."""
        a_impl = impl_flops / (ms / 1e3) / 1e12
        a_meth = method_flops / (ms / 1e3) / 1e12
        return {"achieved_method": a_meth, "frac_method": a_meth / peak_tf,
                "achieved_impl": a_impl, "frac_impl": a_impl / peak_tf}

    form = 1 if args.mode == "fast" else 0  # the factor the kernels run in: U-D fast, square root deterministic
    bwd_f = frac2(flops.backward_flops(lengths, form), flops.method_backward_flops(lengths), bwd_ms)
    fa_f = frac2(flops.fit_adjoint_flops(lengths, form), flops.method_fit_adjoint_flops(lengths), step_ms)
    fit_f = frac2(flops.fit_flops(lengths, form), flops.method_fit_flops(lengths), plain_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "roofline": {"bound": "alu", "achieved": bwd_f["achieved_method"], "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": bwd_f["frac_method"], "traffic": _traffic("backward_" + args.mode),
                     "kernel": "backward_kernel", "launch_ms": bwd_ms,
                     "frac_impl": bwd_f["frac_impl"], "achieved_impl": bwd_f["achieved_impl"],
                     "count": "achieved/frac: method count (480 flop per cluster for the fit, x2.5 for the reverse); "
                              "*_impl: the form as implemented (flops.py; fast mode: U-D)",
                     "peak_source": "measured on this GPU: FMA-chain microbenchmark (fp32_peak)"},
        "fit_adjoint": {"tracks_per_s": value, "ms": step_ms, "fit_ms": fit_rec_ms, "backward_ms": bwd_ms, **fa_f},
        "plain_fit": {"tracks_per_s": fr.n_tracks / (plain_ms / 1e3), "ms": plain_ms,
                      "hits_per_s": fr.n_tracks / (plain_ms / 1e3) * mhits, **fit_f,
                      "traffic": _traffic("fit_" + args.mode)},
        "hits_per_s": value * mhits,
        "e2e": e2e,
        "gpu_launches": 4 * args.steps,
        "clocks": clocks,
        "config": {"workload": WORKLOAD, "step": "fit with checkpoints + adjoint (gradients w.r.t. alignment and seeds)",
                   "mode": args.mode, "tracks": fr.n_tracks, "hits": fr.n_hits, "mean_hits_per_track": mhits,
                   "l2": "inputs larger than L2 (clusters %.0f MB > 126 MB), no flush" % (10 * fr.n_hits / 1e6),
                   "fitted_fraction": float(np.mean(ndf > 0))},
        "fp32_peak": peak,
    }
    if det is not None:
        dfa_ms = det["fit_ms"] + det["backward_ms"]
        line["deterministic"] = {
            "plain_fit": {"tracks_per_s": fr.n_tracks / (det["plain_fit_ms"] / 1e3), "ms": det["plain_fit_ms"],
                          "vs_fast": det["plain_fit_ms"] / plain_ms,
                          **frac2(flops.fit_flops(lengths), flops.method_fit_flops(lengths), det["plain_fit_ms"])},
            "fit_adjoint": {"tracks_per_s": fr.n_tracks / (dfa_ms / 1e3), "ms": dfa_ms, "fit_ms": det["fit_ms"],
                            "backward_ms": det["backward_ms"], "vs_fast": dfa_ms / step_ms,
                            "backward_vs_fast": det["backward_ms"] / bwd_ms},
            "paper_slowdown": "1.5-10x (Sec. 2, the deterministic mode of the whole reconstruction)",
            "note": "no FMA contraction: the deterministic kernels' ceiling is half the FMA peak"}
    if sqrt_form is not None:
        sq_fa = sqrt_form["fit_ms"] + sqrt_form["backward_ms"]
        line["square_root_form"] = {
            "plain_fit": {"ms": sqrt_form["plain_fit_ms"], "vs_u_d": sqrt_form["plain_fit_ms"] / plain_ms,
                          **frac2(flops.fit_flops(lengths, 0), flops.method_fit_flops(lengths),
                                  sqrt_form["plain_fit_ms"])},
            "fit_adjoint": {"tracks_per_s": fr.n_tracks / (sq_fa / 1e3), "ms": sq_fa, "fit_ms": sqrt_form["fit_ms"],
                            "backward_ms": sqrt_form["backward_ms"], "vs_u_d": sq_fa / step_ms},
            "note": "fast mode with the square-root factor and Potter's updates (the deterministic mode's "
                    "sequence) in place of U-D and Bierman's"}
    line["plain_fit"]["e2e"] = e2e_plain
    sm_f = flops.smooth_flops(lengths) / (smooth_ms / 1e3) / 1e12
    line["smoother"] = {"tracks_per_s": fr.n_tracks / (smooth_ms / 1e3), "clusters_per_s": fr.n_hits / (smooth_ms / 1e3),
                        "ms": smooth_ms, "frac_impl": sm_f / peak_tf,
                        "states": {"ms": states_ms, "clusters_per_s": fr.n_hits / (states_ms / 1e3)},
                        "reject": {"ms": reject_ms, "clusters_per_s": fr.n_hits / (reject_ms / 1e3),
                                   "cut": 16.0, "kept_fraction": reject_kept / fr.n_hits,
                                   "bytes_per_cluster": 24, "achieved_gbs": 24 * fr.n_hits / (reject_ms / 1e3) / 1e9}}
    line["plain_fit"]["field_map"] = {"tracks_per_s": fr.n_tracks / (fld_ms / 1e3), "ms": fld_ms,
                                      "field": "Bz (1 + 0.3 (r/250)^2 - 0.2 (z/250)^2)"}
    line["plain_fit"]["material"] = {"tracks_per_s": fr.n_tracks / (mat_ms / 1e3), "ms": mat_ms,
                                     "material": "TPC gas layer at every row"}
    for key, per_ in (("material", mat_fa_per), ("field_map", fld_fa_per)):
        f_ms = statistics.mean(p[0] for p in per_)
        b_ms = statistics.mean(p[1] for p in per_)
        line["fit_adjoint"][key] = {"tracks_per_s": fr.n_tracks / ((f_ms + b_ms) / 1e3), "fit_ms": f_ms,
                                    "backward_ms": b_ms}
    if rtc is not None:
        line["plain_fit"]["rtc"] = {"tracks_per_s": fr.n_tracks / (rtc["ms"] / 1e3), "ms": rtc["ms"],
                                    "first_call_s": rtc["first_call_s"]}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(fr)
    fitter.close()
    if not args.no_extra and world == 1:
        del dev, out
        torch.cuda.empty_cache()
        line["batched_frames"] = run_batched_frames(args, tf, torch, synth, flops, peak_tf)
        line["alignment_loop"] = run_alignment_loop(args, tf, torch, synth)
        if "cpu_baseline" in line:
            # one iteration = fit + gradient of every track: the oracle's rate on
            # the time-frame sample, extrapolated to the loop's tracks
            n_al = args.align_tracks
            line["alignment_loop"]["cpu_baseline"] = {
                "value": line["cpu_baseline"]["value"], "unit": UNIT, "kind": "oracle",
                "cores": line["cpu_baseline"]["cores"],
                "extrapolated_s_per_iteration": n_al / line["cpu_baseline"]["value"],
                "note": "fit + forward-mode gradient rate of the time-frame sample (same track distributions), "
                        "extrapolated to the loop's tracks"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
