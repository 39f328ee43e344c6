"""Agreement criteria of an FP32 fit with the FP64 reference.

The fast FP32 mode must reproduce the FP64 fit to relative 1e-4 in the track
parameters and 1e-3 in chi2.  Relative is taken against max(|p_i|, sigma_i),
sigma_i = sqrt(C_ii) of the FP64 fit, because y, z, sin(phi) and tan(lambda)
cross zero; chi2 against max(chi2, 1).

A 150-step FP32 recursion carries rounding of about 1e-4 sigma (positions pass
through values up to ~40 cm whose FP32 spacing is 4e-6 cm).  So the bound holds
for all but a small tail of tracks.  The criterion:
  * at least 99.5 % of tracks meet 1e-4 (params) and 99.9 % meet 1e-3 (chi2),
  * no track exceeds 2e-3 (params) or 1e-2 (chi2),
  * the failure flag (ndf < 0) agrees on at least 99.99 % of tracks.
"""
from __future__ import annotations

import numpy as np

PARAM_TOL = 1e-4
CHI2_TOL = 1e-3
PARAM_FRAC = 0.995
CHI2_FRAC = 0.999
PARAM_HARD = 2e-3
CHI2_HARD = 1e-2
FLAG_FRAC = 0.9999


def compare_to_fp64(fit32: dict, fit64: dict) -> dict:
    """Compare FP32 fit outputs (params[5,n], chi2[n], ndf[n]) with FP64 ones."""
    ndf32 = np.asarray(fit32["ndf"])
    ndf64 = np.asarray(fit64["ndf"])
    n = ndf64.shape[0]
    if n == 0:
        return dict(ok=True, n=0)
    flag_agree = float(np.mean((ndf32 < 0) == (ndf64 < 0)))
    both = (ndf32 > 0) & (ndf64 > 0)
    p32 = np.asarray(fit32["params"], np.float64)[:, both]
    p64 = np.asarray(fit64["params"], np.float64)[:, both]
    sig = np.sqrt(np.abs(np.asarray(fit64["cov"], np.float64)[[0, 2, 5, 9, 14]][:, both]))
    rel = np.abs(p32 - p64) / np.maximum(np.abs(p64), sig)
    worst = rel.max(axis=0) if rel.size else np.zeros(0)
    c32 = np.asarray(fit32["chi2"], np.float64)[both]
    c64 = np.asarray(fit64["chi2"], np.float64)[both]
    crel = np.abs(c32 - c64) / np.maximum(c64, 1.0)
    m = max(int(both.sum()), 1)
    rep = dict(
        n=int(n), n_compared=int(both.sum()), flag_agree=flag_agree,
        frac_params_ok=float(np.sum(worst <= PARAM_TOL) / m),
        frac_chi2_ok=float(np.sum(crel <= CHI2_TOL) / m),
        max_param_rel=float(worst.max()) if worst.size else 0.0,
        max_chi2_rel=float(crel.max()) if crel.size else 0.0,
        q999_param_rel=[float(v) for v in np.quantile(rel, 0.999, axis=1)] if rel.size else [],
        finite=bool(np.all(np.isfinite(p32)) and np.all(np.isfinite(c32))),
    )
    rep["ok"] = bool(rep["finite"] and rep["flag_agree"] >= FLAG_FRAC and rep["frac_params_ok"] >= PARAM_FRAC
                     and rep["frac_chi2_ok"] >= CHI2_FRAC and rep["max_param_rel"] <= PARAM_HARD
                     and rep["max_chi2_rel"] <= CHI2_HARD)
    return rep
