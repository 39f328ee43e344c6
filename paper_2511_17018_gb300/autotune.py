"""Autotuner of the fit's launch configuration.

Sweeps lanes per track (tracks per warp = 32 / lanes), clusters staged per
refill (rows per stage) and warps per block, with and without the length
ordering, timing tpcfit_fit (or tpcfit_fit_frames) with CUDA events on a
sample of the workload whose length histogram matches the whole.  Shapes the
library does not provide are skipped (tpcfit_set_config answers EINVAL): one
lane per track comes in six (rows per stage, warps) shapes, 2 to 32 lanes per
track in (4, 24).  The best configuration is cached per (mode, GPU name,
length-histogram bucket, size bucket) in a JSON file, with the fastest time
of every lanes-per-track value.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

from . import tpcfit as tf

LANES = (1, 2, 4, 8, 16, 32)       # tracks per warp 32, 16, 8, 4, 2, 1
ROWS_PER_STAGE = (4, 8, 16)
WARPS = (8, 12, 16, 24)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build", "autotune.json")


def bucket_key(mode: str, lengths, n_tracks: int) -> str:
    """Cache key: mode, GPU, mean-length bucket (width 16) and log2 size bucket."""
    gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    mean_len = float(np.mean(lengths)) if len(lengths) else 0.0
    return f"{mode}|{gpu}|len{int(mean_len // 16) * 16}|n2^{int(np.log2(max(n_tracks, 1)))}"


def candidates():
    for lanes in LANES:
        for rps in ROWS_PER_STAGE:
            for warps in WARPS:
                for srt in (True, False):
                    yield lanes, rps, warps, srt


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def tune(fitter, dev: dict, lengths, mode: str = "fast", reps: int = 5, cache_path: str | None = DEFAULT_CACHE,
         fit_call=None, force: bool = False) -> dict:
    """Pick the fastest configuration for this workload and set it on `fitter`.

    dev: device inputs (as tf.frame_to_device); fit_call(out) overrides the
    timed call (e.g. a batched-frames fit).  Returns the chosen entry."""
    n = int(dev["offsets"].numel()) - 1
    key = bucket_key(mode, lengths, n)
    cache = load_cache(cache_path) if cache_path else {}
    if key in cache and not force:
        ent = cache[key]
        fitter.set_config(ent["lanes_per_track"], ent["rows_per_stage"], ent["warps_per_block"], ent["sort_by_length"])
        return ent
    fitter.set_mode(mode == "det")
    out = tf.empty_outputs(n, dev["y"].device)
    call = fit_call or (lambda: fitter.fit(dev, out))
    results = []
    t0 = time.time()
    for lanes, rps, warps, srt in candidates():
        try:
            fitter.set_config(lanes, rps, warps, srt)
        except tf.TpcfitError:
            continue
        ms = _time(call, reps)
        results.append(dict(lanes_per_track=lanes, rows_per_stage=rps, warps_per_block=warps, sort_by_length=srt,
                            ms=ms))
    best = min(results, key=lambda r: r["ms"])
    by_lanes = {}
    for r in results:
        k = str(r["lanes_per_track"])
        if k not in by_lanes or r["ms"] < by_lanes[k]["ms"]:
            by_lanes[k] = {kk: r[kk] for kk in ("rows_per_stage", "warps_per_block", "sort_by_length", "ms")}
    best = dict(best, key=key, tried=len(results), sweep_s=time.time() - t0,
                table=sorted(results, key=lambda r: r["ms"])[:8], by_lanes=by_lanes)
    fitter.set_config(best["lanes_per_track"], best["rows_per_stage"], best["warps_per_block"],
                      best["sort_by_length"])
    if cache_path:
        cache[key] = best
        save_cache(cache, cache_path)
    return best


def sample_tracks(frame, fraction: float = 0.01, minimum: int = 20000, seed: int = 0):
    """A track sample (index array) with the frame's length histogram: a seeded
    uniform draw of max(fraction * N, minimum) tracks (all if fewer)."""
    n = frame.n_tracks
    m = min(n, max(int(fraction * n), minimum))
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, m, replace=False))
