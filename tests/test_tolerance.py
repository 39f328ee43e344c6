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
    # a tail between 1e-4 and the hard bound: 1 track in 10,000 passes, 2 fail
    for k, ok in ((1, True), (2, False)):
        got = _copy(ref)
        got["params"][2, 200:200 + k] *= 1.0 + 3.0 * tol.PARAM_TOL
        assert tol.compare_to_fp64(got, ref)["ok"] is ok, k


def test_chi2_flag_and_finiteness_bounds():
    ref = _ref()
    got = _copy(ref)
    got["chi2"][7] *= 1.0 + 2.0 * tol.CHI2_HARD
    assert not tol.compare_to_fp64(got, ref)["ok"]
    got = _copy(ref)
    got["chi2"][:2] *= 1.0 + 3.0 * tol.CHI2_TOL   # 2 of 10,000 past 1e-3: beyond the 0.01 % allowed
    assert not tol.compare_to_fp64(got, ref)["ok"]
    got = _copy(ref)
    got["chi2"][:1] *= 1.0 + 3.0 * tol.CHI2_TOL   # 1 of 10,000: allowed
    assert tol.compare_to_fp64(got, ref)["ok"]
    got = _copy(ref)
    got["ndf"][3] = -1                           # one flag in 10,000 differs: at the 99.99 % bound
    assert tol.compare_to_fp64(got, ref)["ok"]
    got["ndf"][4] = -1                           # two: past it
    assert not tol.compare_to_fp64(got, ref)["ok"]
    got = _copy(ref)
    got["params"][1, 9] = np.nan
    assert not tol.compare_to_fp64(got, ref)["ok"]


def test_covariance_bounds():
    # a covariance element is judged against sqrt(C_ii C_jj)
    ref = _ref()
    ref["cov"][1] = 0.3 * 0.01                    # C_10 of correlation 0.3
    got = _copy(ref)
    got["cov"][1, 10] += 0.5 * tol.COV_TOL * 0.01  # inside 1e-4 of sqrt(C00 C11)
    assert tol.compare_to_fp64(got, ref)["ok"]
    got = _copy(ref)
    got["cov"][14, 11] *= 1.0 + 2.0 * tol.COV_HARD  # one element past the hard bound
    assert not tol.compare_to_fp64(got, ref)["ok"]
    got = _copy(ref)
    got["cov"][5, 20:22] *= 1.0 + 3.0 * tol.COV_TOL  # two tracks past 1e-4
    assert not tol.compare_to_fp64(got, ref)["ok"]
    got = _copy(ref)
    got["cov"][9, 30] = np.nan
    assert not tol.compare_to_fp64(got, ref)["ok"]


def test_gradient_errors_floor():
    ref = np.array([1.0, -2.0, 1e-9, 0.5])
    got = ref * (1 + 1e-6)
    got[2] = 1e-9 + 1e-9                          # 100 % off, but far below the 1e-3 floor of max|g|
    e = tol.gradient_errors(got, ref)
    assert e["max"] < 1e-5
    got[1] = -2.0 * (1 + 1e-4)
    assert tol.gradient_errors(got, ref)["max"] > 9e-5


def test_small_samples_allow_one_miss():
    ref = _ref(n=1000)
    got = _copy(ref)
    got["params"][3, 500] *= 1.0 + 3.0 * tol.PARAM_TOL
    assert tol.compare_to_fp64(got, ref)["ok"]
    got["params"][3, 501] *= 1.0 + 3.0 * tol.PARAM_TOL
    assert not tol.compare_to_fp64(got, ref)["ok"]
