"""The fast-mode agreement criterion rejects what it should (CPU).

Every fast-mode parity test goes through tolerance.compare_to_fp64, so its
bounds are checked here on constructed outputs: each planted deviation just
past a bound fails, one just inside it passes."""
import numpy as np

from paper_2511_17018_gb300 import tolerance as tol


def _ref(n=10000, seed=0):
    rng = np.random.default_rng(seed)
    params = rng.normal(0.0, 1.0, (5, n))
    params[:, :100] = 0.0                        # parameters at zero: the scale is sigma
    cov = np.zeros((15, n))
    for d, s in zip((0, 2, 5, 9, 14), (0.01, 0.01, 1e-6, 1e-6, 1e-4)):
        cov[d] = s
    chi2 = rng.chisquare(100, n)
    ndf = np.full(n, 100, np.int32)
    return dict(params=params, cov=cov, chi2=chi2, ndf=ndf)


def _copy(ref):
    return {k: v.copy() for k, v in ref.items()}


def test_identical_outputs_pass():
    ref = _ref()
    rep = tol.compare_to_fp64(_copy(ref), ref)
    assert rep["ok"] and rep["max_param_rel"] == 0.0


def test_parameter_bounds():
    ref = _ref()
    n = ref["ndf"].size
    # a parameter at zero is compared against sigma: 0.5 sigma_rel of 1e-4 passes
    got = _copy(ref)
    got["params"][0, 5] = 0.5e-4 * 0.1
    assert tol.compare_to_fp64(got, ref)["ok"]
    # one track beyond the hard bound fails
    got = _copy(ref)
    got["params"][4, 200] *= 1.0 + 2.5 * tol.PARAM_HARD
    assert not tol.compare_to_fp64(got, ref)["ok"]
    # a tail between 1e-4 and the hard bound: 0.3 % of tracks pass, 1 % fail
    for frac, ok in ((0.003, True), (0.01, False)):
        got = _copy(ref)
        k = int(frac * n)
        got["params"][2, 200:200 + k] *= 1.0 + 5.0 * tol.PARAM_TOL
        assert tol.compare_to_fp64(got, ref)["ok"] is ok, frac


def test_chi2_flag_and_finiteness_bounds():
    ref = _ref()
    got = _copy(ref)
    got["chi2"][7] *= 1.0 + 2.0 * tol.CHI2_HARD
    assert not tol.compare_to_fp64(got, ref)["ok"]
    got = _copy(ref)
    got["chi2"][: int(0.002 * got["chi2"].size)] *= 1.0 + 5.0 * tol.CHI2_TOL   # 0.2 % > the 0.1 % allowed
    assert not tol.compare_to_fp64(got, ref)["ok"]
    got = _copy(ref)
    got["ndf"][3] = -1                           # one flag in 10,000 differs: at the 99.99 % bound
    assert tol.compare_to_fp64(got, ref)["ok"]
    got["ndf"][4] = -1                           # two: past it
    assert not tol.compare_to_fp64(got, ref)["ok"]
    got = _copy(ref)
    got["params"][1, 9] = np.nan
    assert not tol.compare_to_fp64(got, ref)["ok"]
