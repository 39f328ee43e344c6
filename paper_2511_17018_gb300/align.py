"""Alignment recovery: fit + adjoint + Adam on the 36 x 152 x 2 offsets, on the device.

Each iteration uploads the current offset estimate to the fitter, fits every
track with checkpoints, runs the adjoint of L = mean chi2 over fitted tracks
and applies one Adam step (Kingma & Ba, 2015) to the offsets.  The iteration
is captured in a CUDA graph once and replayed.  The loop's state (offsets,
Adam moments, step count) can be written to a file every few iterations and
read back to resume; the file is replaced atomically, so an interrupted run
leaves the previous checkpoint intact.

Offsets that a helix absorbs cannot be recovered from chi2: per sector,
dy_r = a + b X_r + c X_r^2 and dz_r = a' + b' X_r move every cluster of that
sector along a curve that the track parameters (y, sin phi, q/pt) and (z,
tan lambda) follow.  `recovery` therefore reports the RMS of the estimate's
error both raw and after projecting out these five modes per sector.
"""
from __future__ import annotations

import os

import numpy as np
import torch

from . import tpcfit as tf


class AlignmentLoop:
    def __init__(self, fitter, dev: dict, lr: float = 5e-3, betas=(0.9, 0.999), eps: float = 1e-8,
                 use_graph: bool = True):
        self.f, self.dev = fitter, dev
        n = int(dev["offsets"].numel()) - 1
        device = dev["y"].device
        self.n = n
        self.lr, self.b1, self.b2, self.eps = lr, betas[0], betas[1], eps
        self.d = torch.zeros(36 * 152 * 2, dtype=torch.float32, device=device)
        self.m = torch.zeros_like(self.d)
        self.v = torch.zeros_like(self.d)
        self.t = torch.zeros((), dtype=torch.float32, device=device)
        self.b1t = torch.tensor(self.b1, dtype=torch.float32, device=device)  # made before any capture
        self.b2t = torch.tensor(self.b2, dtype=torch.float32, device=device)
        self.loss = torch.zeros((), dtype=torch.float32, device=device)
        self.out = tf.empty_outputs(n, device)
        self.ga = torch.empty_like(self.d)
        self.gs = torch.empty((5, n), dtype=torch.float32, device=device)
        self.g = torch.empty(n, dtype=torch.float32, device=device)
        self.graph = None
        fitter.set_record(True)
        tf.tpcfit_reserve(fitter.h, n, int(dev["y"].numel()))
        if use_graph:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                self._iteration()           # warm-up: scratch, constants, allocator pools
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            self.reset()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._iteration()

    def reset(self):
        for x in (self.d, self.m, self.v, self.t):
            x.zero_()

    # ---- checkpoint / resume
    STATE_KEYS = ("d", "m", "v", "t")

    def state_dict(self) -> dict:
        """Offsets, Adam moments and step count (host copies) with the settings."""
        sd = {k: getattr(self, k).detach().cpu().clone() for k in self.STATE_KEYS}
        sd.update(lr=self.lr, betas=(self.b1, self.b2), eps=self.eps, n_tracks=self.n)
        return sd

    def load_state_dict(self, sd: dict):
        """Copy a saved state into the loop's buffers in place (the captured
        graph keeps reading the same device memory).  The settings must match."""
        if (sd["lr"], tuple(sd["betas"]), sd["eps"]) != (self.lr, (self.b1, self.b2), self.eps):
            raise ValueError("checkpoint was written with other Adam settings")
        if sd["n_tracks"] != self.n:
            raise ValueError("checkpoint was written for another track sample")
        for k in self.STATE_KEYS:
            dst = getattr(self, k)
            src = sd[k]
            if tuple(src.shape) != tuple(dst.shape):
                raise ValueError(f"checkpoint entry {k} has shape {tuple(src.shape)}, expected {tuple(dst.shape)}")
            dst.copy_(src.to(dst.device, dst.dtype))

    def save(self, path: str):
        save_state(path, self.state_dict())

    def load(self, path: str):
        self.load_state_dict(load_state(path))

    @property
    def iteration(self) -> int:
        return int(self.t.item())

    def _iteration(self):
        tf.tpcfit_set_alignment(self.f.h, self.d)
        self.f.fit(self.dev, self.out)
        ok = (self.out["ndf"] > 0).to(torch.float32)
        cnt = ok.sum().clamp(min=1.0)
        torch.div(ok, cnt, out=self.g)
        self.loss.copy_(torch.nan_to_num(self.out["chi2"], nan=0.0).mul(ok).sum() / cnt)
        tf.tpcfit_fit_backward(self.f.h, self.dev["y"], self.dev["z"], self.dev["rowsec"], self.dev["offsets"],
                               self.out["ndf"], self.g, self.ga, self.gs)
        # Adam with bias correction (device-side step counter, graph-capturable)
        self.t.add_(1.0)
        self.m.mul_(self.b1).add_(self.ga, alpha=1.0 - self.b1)
        self.v.mul_(self.b2).addcmul_(self.ga, self.ga, value=1.0 - self.b2)
        bc1 = 1.0 - torch.pow(self.b1t, self.t)
        bc2 = 1.0 - torch.pow(self.b2t, self.t)
        step = (self.m / bc1) / (torch.sqrt(self.v / bc2) + self.eps)
        self.d.sub_(step, alpha=self.lr)

    def step(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._iteration()
        return self.loss

    def run(self, iters: int, checkpoint: str | None = None, every: int = 0):
        """`iters` iterations; with `checkpoint` and `every` > 0 the state is
        saved to that file after every `every`-th iteration (counted from the
        start of the whole run, resumed runs included) and after the last."""
        losses = []
        start = self.iteration if checkpoint else 0
        for i in range(iters):
            losses.append(self.step().clone())
            if checkpoint and every > 0 and ((start + i + 1) % every == 0 or i == iters - 1):
                self.save(checkpoint)
        torch.cuda.synchronize()
        return torch.stack(losses).cpu().numpy()


def save_state(path: str, sd: dict):
    """Write a loop state to `path` through a temporary file and a rename."""
    tmp = f"{path}.tmp{os.getpid()}"
    torch.save(sd, tmp)
    os.replace(tmp, path)


def load_state(path: str) -> dict:
    return torch.load(path, map_location="cpu", weights_only=True)


def weak_mode_basis(row_x):
    """Per sector: columns spanning the unobservable offsets (dy: 1, X, X^2; dz: 1, X)."""
    X = np.asarray(row_x, np.float64)
    Xn = (X - X.mean()) / X.std()
    return np.stack([np.ones_like(Xn), Xn, Xn * Xn], axis=1), np.stack([np.ones_like(Xn), Xn], axis=1)


def recovery(d_est, d_true, row_x):
    """RMS of (estimate - truth) over all 10,944 offsets, raw and with the five
    weak modes per sector projected out."""
    err = np.asarray(d_est, np.float64).reshape(36, 152, 2) - np.asarray(d_true, np.float64).reshape(36, 152, 2)
    By, Bz = weak_mode_basis(row_x)
    proj = err.copy()
    for s in range(36):
        for c, B in ((0, By), (1, Bz)):
            coef, *_ = np.linalg.lstsq(B, err[s, :, c], rcond=None)
            proj[s, :, c] -= B @ coef
    return float(np.sqrt(np.mean(err ** 2))), float(np.sqrt(np.mean(proj ** 2)))
