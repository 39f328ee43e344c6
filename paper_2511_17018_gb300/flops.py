"""Algorithmic FP32 operation counts of the fit and its adjoint (roofline accounting).

Counted from the formula list of one step as the kernels evaluate it: every
add, subtract and multiply is one operation (a fused multiply-add counts as
two), every division, reciprocal and square root one.  Square-root form: a
step = rotation-free prediction (79, with the d(path)/dk series that
single-row steps use) + transport L <- J L (60) + two Potter scalar updates
(2 x 128) + the alignment subtraction (2).  U-D form: the same prediction +
transport U <- J U (16) + Bierman's updates of y (85) and z (75) + 2.  The
first cluster of a pass has no prediction or transport.  The output
covariance costs 135 per track from L, 70 from U and D.  form: 0 square
root, 1 U-D.
"""
from __future__ import annotations

import numpy as np

PREDICT = 79
TRANSPORT = 60
SCALAR_UPDATE = 128
MEAS = 2
STEP = PREDICT + TRANSPORT + 2 * SCALAR_UPDATE + MEAS          # 397
FIRST = 2 * SCALAR_UPDATE + MEAS                               # 258
OUTPUT = 135
UD_TRANSPORT = 16
UD_UPDATE = (85, 75)
UD_STEP = PREDICT + UD_TRANSPORT + sum(UD_UPDATE) + MEAS       # 257
UD_FIRST = sum(UD_UPDATE) + MEAS                               # 162
UD_OUTPUT = 70


def fit_flops(lengths, form: int = 0) -> float:
    """Algorithmic flops of fitting tracks with the given cluster counts (both passes)."""
    n = np.asarray(lengths, dtype=np.int64)
    n = n[n >= 1]
    step, first, out = (UD_STEP, UD_FIRST, UD_OUTPUT) if form == 1 else (STEP, FIRST, OUTPUT)
    return float(np.sum(2 * ((n - 1) * step + first) + out))


def fit_bytes(lengths) -> float:
    """Algorithmic DRAM bytes: clusters read once (10 B), per track offsets (4),
    seeds (20), outputs (5 + 15 + 1 + 1 words = 88)."""
    n = np.asarray(lengths, dtype=np.int64)
    return float(10 * n.sum() + (4 + 20 + 88) * n.shape[0])


# Reverse sweep (adjoint), counted from the formula list of the hand-written
# reverse of each forward piece: a Potter scalar update (268), the transport
# L <- J L (120) and the prediction with its Jacobian (150); in U-D form
# Bierman's updates of y (260) and z (226, their partial gain sums recomputed
# in the forward's order included) and the transport U <- J U (20).
# Recomputation of forward values (checkpoint segments, per-step
# intermediates) is overhead and is not counted.
REV_SCALAR_UPDATE = 268
REV_TRANSPORT = 120
REV_PREDICT = 150
REV_STEP = REV_PREDICT + REV_TRANSPORT + 2 * REV_SCALAR_UPDATE   # 806
REV_FIRST = 2 * REV_SCALAR_UPDATE                                 # 536
UD_REV_UPDATE = (260, 226)
UD_REV_TRANSPORT = 20
UD_REV_STEP = REV_PREDICT + UD_REV_TRANSPORT + sum(UD_REV_UPDATE)  # 656
UD_REV_FIRST = sum(UD_REV_UPDATE)                                   # 486


def backward_flops(lengths, form: int = 0) -> float:
    """Algorithmic flops of the reverse sweep over both passes."""
    n = np.asarray(lengths, dtype=np.int64)
    n = n[n >= 1]
    step, first = (UD_REV_STEP, UD_REV_FIRST) if form == 1 else (REV_STEP, REV_FIRST)
    return float(np.sum(2 * ((n - 1) * step + first)))


def fit_adjoint_flops(lengths, form: int = 0) -> float:
    return fit_flops(lengths, form) + backward_flops(lengths, form)


# Two-filter smoother, per cluster: the outward filter it runs (a fit step,
# STEP; FIRST at the first cluster) and the square-root combination of the two
# predictions (Householder QR of the stacked 10x5 factors with the two 2x10
# row blocks carried along: 1100; the triangular solve 30; the corrections and
# H C H^T 54; R and chi2 20).  Recomputing the inward predictions from the
# checkpoints is overhead and is not counted.
SMOOTH_COMBINE = 1100 + 30 + 54 + 20


def smooth_flops(lengths) -> float:
    """Algorithmic flops of the smoother over all clusters of fitted tracks."""
    n = np.asarray(lengths, dtype=np.int64)
    n = n[n >= 1]
    return float(np.sum((n - 1) * STEP + FIRST + n * SMOOTH_COMBINE))


# The method's count (the textbook covariance-form filter, estimated per step
# and pass: propagation ~20, Jacobian ~20, transport ~100, update ~120 -> 240;
# both passes -> 480 per cluster), and the adjoint's reverse sweep at 2.5 times
# the forward (fit + adjoint = 3.5 x fit).  It credits none of the work the
# square-root form and the residual coordinates add, so fractions taken on it
# are the conservative ones.
METHOD_STEP = 240
METHOD_REVERSE_FACTOR = 2.5


def method_fit_flops(lengths) -> float:
    """The method's count of the fit: 480 flops per cluster (two passes of 240)."""
    n = np.asarray(lengths, dtype=np.int64)
    return float(2 * METHOD_STEP * n[n >= 1].sum())


def method_backward_flops(lengths) -> float:
    return METHOD_REVERSE_FACTOR * method_fit_flops(lengths)


def method_fit_adjoint_flops(lengths) -> float:
    return (1.0 + METHOD_REVERSE_FACTOR) * method_fit_flops(lengths)
