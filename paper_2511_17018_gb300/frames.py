"""Many time frames in one persistent launch, optionally replayed as a CUDA graph.

FrameBatch concatenates frames (clusters, offsets, seeds) into the layout of
tpcfit_fit_frames and keeps the frame table; GraphedFrameFit captures the call
(ordering kernels + persistent fit) in a CUDA graph once and replays it.
"""
from __future__ import annotations

import numpy as np
import torch

from . import tpcfit as tf


class FrameBatch:
    """Device-resident concatenation of frames.

    frames: list of synth.Frame, or (pool Frame, list of per-frame track index
    arrays) to build frames by sampling tracks from a pool on the device."""

    def __init__(self, y, z, rowsec, offsets, seeds, frame_base):
        self.y, self.z, self.rowsec, self.offsets, self.seeds = y, z, rowsec, offsets, seeds
        self.frame_base = frame_base
        self.n_tracks = int(offsets.numel()) - 1
        self.n_hits = int(y.numel())
        self.n_frames = int(frame_base.numel()) - 1

    @staticmethod
    def from_frames(frames, device="cuda"):
        from .synth import concat
        cat = concat(list(frames))
        base = np.concatenate([[0], np.cumsum([f.n_tracks for f in frames])]).astype(np.int64)
        d = tf.frame_to_device(cat, device)
        return FrameBatch(d["y"], d["z"], d["rowsec"], d["offsets"], d["seeds"],
                          torch.from_numpy(base).to(device))

    @staticmethod
    def from_pool(pool, picks, device="cuda"):
        """Frames made of pool tracks (gathered on the device): frame f holds the
        tracks picks[f] of `pool`, in that order."""
        d = tf.frame_to_device(pool, device)
        idx = torch.from_numpy(np.concatenate(picks).astype(np.int64)).to(device)
        off = d["offsets"].to(torch.int64)
        lens = off[1:] - off[:-1]
        tl = lens[idx]
        new_off = torch.zeros(idx.numel() + 1, dtype=torch.int64, device=device)
        torch.cumsum(tl, 0, out=new_off[1:])
        total = int(new_off[-1].item())
        if total >= 2**31:
            raise ValueError("batched frames exceed int32 cluster offsets")
        # cluster gather index: for output position j in track k -> off[idx[k]] + (j - new_off[k])
        owner = torch.repeat_interleave(torch.arange(idx.numel(), device=device), tl)
        src = off[idx][owner] + (torch.arange(total, device=device) - new_off[:-1][owner])
        base = np.concatenate([[0], np.cumsum([len(p) for p in picks])]).astype(np.int64)
        return FrameBatch(d["y"][src].contiguous(), d["z"][src].contiguous(), d["rowsec"][src].contiguous(),
                          new_off.to(torch.int32), d["seeds"][:, idx].contiguous(),
                          torch.from_numpy(base).to(device))

    def dev(self):
        return dict(y=self.y, z=self.z, rowsec=self.rowsec, offsets=self.offsets, seeds=self.seeds)


def fit_frames(fitter, batch: FrameBatch, out=None, frame_alignment=None, frame_ready=None, wait_timeout_ns=0,
               stream=None):
    out = out or tf.empty_outputs(batch.n_tracks, batch.y.device)
    tf.tpcfit_fit_frames(fitter.h, batch.y, batch.z, batch.rowsec, batch.offsets, batch.frame_base, batch.seeds,
                         out["params"], out["cov"], out["chi2"], out["ndf"], frame_alignment, frame_ready,
                         wait_timeout_ns, stream)
    return out


class GraphedFrameFit:
    """tpcfit_fit_frames captured once in a CUDA graph; replay() refits the
    batch (whose device buffers may be refilled in place between replays)."""

    def __init__(self, fitter, batch: FrameBatch, frame_alignment=None):
        self.fitter, self.batch, self.fa = fitter, batch, frame_alignment
        self.out = tf.empty_outputs(batch.n_tracks, batch.y.device)
        tf.tpcfit_reserve(fitter.h, batch.n_tracks, batch.n_hits)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            fit_frames(fitter, batch, self.out, frame_alignment)  # warm-up: scratch and constants in place
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            fit_frames(fitter, batch, self.out, frame_alignment)

    def replay(self):
        self.graph.replay()
        return self.out
