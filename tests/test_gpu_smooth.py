"""Two-filter smoother on the GPU against the FP64 oracle (run on a GB300 with -m gpu).

Per cluster the leave-one-out residual, its covariance and chi2 agree with the
oracle's information-form combination within the FP32 tolerance below (the
same FP32-vs-FP64 rounding argument as for the fit: residuals of ~0.1 cm
carried through ~150 steps); the deterministic mode repeats bit for bit; a
displaced cluster is flagged.  The smoothed state and covariance at every
cluster agree with the oracle's two-filter combination, and at the first
cluster equal the kernel's own fit output combined with the seed prior."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2511_17018_gb300 import synth  # noqa: E402
from paper_2511_17018_gb300 import tpcfit as tf  # noqa: E402


def _smooth(fr, det, rps=4, warps=24, srt=True, align=None):
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz, deterministic=det, rows_per_stage=rps, warps_per_block=warps,
                  sort_by_length=srt)
    try:
        if align is not None:
            f.set_alignment(torch.from_numpy(align).cuda())
        f.set_record(True)
        out = f.fit(dev)
        sm = f.smooth(dev, out)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in sm.items()}, out["ndf"].cpu().numpy()
    finally:
        f.close()


def compare(got, ref):
    """Fractions of clusters within tolerance; NaN patterns must agree on all
    but a few clusters (a FP32 step that fails at the |sin phi| limit where
    FP64 does not ends the outward pass one cluster early)."""
    okr, okg = np.isfinite(ref["chi2"]), np.isfinite(got["chi2"])
    both = okr & okg
    sR = np.sqrt(ref["rcov"][both][:, [0, 2]])
    dr = (np.abs(got["resid"][both] - ref["resid"][both]) / sR).max(axis=1)
    rR = ref["rcov"][both]
    dR = np.maximum(np.abs(got["rcov"][both][:, [0, 2]] - rR[:, [0, 2]]).max(axis=1) / rR[:, [0, 2]].min(axis=1),
                    np.abs(got["rcov"][both][:, 1] - rR[:, 1]) / np.sqrt(rR[:, 0] * rR[:, 2]))
    dc = np.abs(got["chi2"][both] - ref["chi2"][both]) / np.maximum(ref["chi2"][both], 1.0)
    return dict(nan_agree=float(np.mean(okr == okg)), n=int(both.sum()),
                resid_ok=float(np.mean(dr < 1e-3)), resid_max=float(dr.max()),
                rcov_ok=float(np.mean(dR < 1e-3)), rcov_max=float(dR.max()),
                chi2_ok=float(np.mean(dc < 1e-3)), chi2_max=float(dc.max()))


@pytest.mark.parametrize("det", [False, True])
def test_smoother_matches_fp64_oracle(det):
    d = synth.alignment_offsets(3)
    fr = synth.generate(20000, 3, drop_p=0.05, cap_lengths=True, d_true=d)
    got, ndf = _smooth(fr, det, align=d)
    ref = oracle.smooth(fr, align=d)
    rep = compare(got, ref)
    print(rep)
    assert rep["nan_agree"] > 0.9999, rep
    assert rep["resid_ok"] > 0.999 and rep["rcov_ok"] > 0.999 and rep["chi2_ok"] > 0.999, rep
    assert rep["resid_max"] < 0.05 and rep["rcov_max"] < 0.05 and rep["chi2_max"] < 0.1, rep
    # every cluster of a track without a fit is NaN
    off = fr.offsets
    for i in np.nonzero(ndf <= 0)[0]:
        assert np.all(np.isnan(got["chi2"][off[i]:off[i + 1]]))


def test_deterministic_smoother_repeats_bit_for_bit():
    fr = synth.generate(5000, 4, drop_p=0.05, cap_lengths=True)
    base, _ = _smooth(fr, True)
    for rps, warps, srt in ((8, 16, False), (4, 12, True)):
        got, _ = _smooth(fr, True, rps, warps, srt)
        for k in base:
            assert np.array_equal(got[k].view(np.int32), base[k].view(np.int32)), (k, rps, warps, srt)


def test_smoother_flags_a_displaced_cluster():
    # a cluster moved by 1 cm (10 sigma) in every track: the GPU flags
    # (chi2 above the 2-dof 1e-3 quantile, 13.8) the clusters the oracle flags
    fr = synth.generate(2000, 31, drop_p=0.05, cap_lengths=True)
    off = fr.offsets
    moved = off[:-1] + np.diff(off) // 2
    fr.y = fr.y.copy()
    fr.y[moved] += np.float32(1.0)
    got, ndf = _smooth(fr, False)
    ref = oracle.smooth(fr)
    with np.errstate(invalid="ignore"):
        fg, fo = got["chi2"] > 13.8, ref["chi2"] > 13.8
    assert np.mean(fg == fo) > 0.9999
    fitted = ndf > 0
    assert np.mean(fg[moved[fitted]]) > 0.995


def test_smoother_needs_a_recorded_fit():
    fr = synth.plain_frame()
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        out = f.fit(dev)                      # recording off
        with pytest.raises(tf.TpcfitError) as e:
            f.smooth(dev, out)
        assert e.value.status == tf.ESTATE
    finally:
        f.close()


def _states(fr, det, align=None, material=None):
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz, deterministic=det)
    try:
        f.set_material(material)
        if align is not None:
            f.set_alignment(torch.from_numpy(align).cuda())
        f.set_record(True)
        out = f.fit(dev)
        sm = f.smooth_states(dev, out)
        again = f.smooth_states(dev, out)
        torch.cuda.synchronize()
        return ({k: v.cpu().numpy() for k, v in sm.items()}, {k: v.cpu().numpy() for k, v in again.items()})
    finally:
        f.close()


def compare_states(got, ref):
    """Smoothed states relative to max(|x_i|, sqrt(C_ii)) of the FP64 result
    (the reading of the fit's tolerance: y, z, sin phi and tan lambda cross
    zero), their covariances relative to sqrt(C_ii C_jj); NaN patterns must
    agree on all but a few clusters."""
    okr, okg = np.all(np.isfinite(ref["state"]), axis=1), np.all(np.isfinite(got["state"]), axis=1)
    both = okr & okg
    C = ref["state_cov"][both]
    sig = np.sqrt(C[:, [0, 2, 5, 9, 14]])
    x = ref["state"][both]
    ds = (np.abs(got["state"][both] - x) / np.maximum(np.abs(x), sig)).max(axis=1)
    pk = [(i, j) for i in range(5) for j in range(i + 1)]
    den = np.stack([sig[:, i] * sig[:, j] for i, j in pk], axis=1)
    dc = (np.abs(got["state_cov"][both] - C) / den).max(axis=1)
    return dict(nan_agree=float(np.mean(okr == okg)), n=int(both.sum()), state_ok=float(np.mean(ds < 1e-4)),
                state_max=float(ds.max()), cov_ok=float(np.mean(dc < 1e-3)), cov_max=float(dc.max()))


@pytest.mark.parametrize("det", [False, True])
def test_smoothed_states_match_fp64_oracle(det):
    # the state at every cluster from all clusters of its track, against the
    # oracle's information-form combination of the outward filtered state and
    # the inward prediction; the deterministic mode repeats bit for bit
    d = synth.alignment_offsets(3)
    fr = synth.generate(8000, 13, drop_p=0.05, cap_lengths=True, d_true=d)
    got, again = _states(fr, det, align=d)
    ref = oracle.smooth_states(fr, align=d)
    rep = compare_states(got, ref)
    print(rep)
    assert rep["nan_agree"] > 0.9999 and rep["n"] > 0.99 * fr.n_hits, rep
    assert rep["state_ok"] > 0.999 and rep["cov_ok"] > 0.98, rep
    assert rep["state_max"] < 5e-3 and rep["cov_max"] < 0.1, rep
    if det:
        for k in got:
            assert np.array_equal(got[k].view(np.int32), again[k].view(np.int32))


def test_smoothed_states_with_material():
    fr = synth.generate(4000, 14, drop_p=0.05, cap_lengths=True)
    fr.material = synth.TPC_GAS
    got, _ = _states(fr, False, material=synth.TPC_GAS)
    rep = compare_states(got, oracle.smooth_states(fr))
    print(rep)
    assert rep["nan_agree"] > 0.9999 and rep["state_ok"] > 0.999 and rep["cov_ok"] > 0.98, rep


def test_smoothed_state_at_the_first_cluster_is_the_fit_with_the_seed_prior():
    # at the first cluster the smoothed state holds every cluster and the
    # outward pass's seed prior (seed, 100 I): the kernel's own fit output
    # combined with that prior in information form, up to FP32 rounding
    fr = synth.generate(2000, 15, drop_p=0.05, cap_lengths=True)
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        f.set_record(True)
        out = f.fit(dev)
        sm = f.smooth_states(dev, out)
        torch.cuda.synchronize()
        st = sm["state"].cpu().numpy().astype(np.float64)
        params = out["params"].cpu().numpy().astype(np.float64)
        cov = out["cov"].cpu().numpy().astype(np.float64)
        ndf = out["ndf"].cpu().numpy()
    finally:
        f.close()
    ok = ndf > 0
    assert ok.mean() > 0.95
    first = fr.offsets[:-1][ok]
    If = np.linalg.inv(np.moveaxis(oracle.unpack(cov[:, ok]), -1, 0))
    Cs = np.linalg.inv(If + np.eye(5) / 100.0)
    xs = np.einsum("nij,nj->ni", Cs, np.einsum("nij,nj->ni", If, params[:, ok].T)
                   + fr.seeds[:, ok].T.astype(np.float64) / 100.0)
    sig = np.sqrt(np.einsum("nii->ni", Cs))
    d = np.abs(st[first] - xs) / np.maximum(np.abs(xs), sig)
    print(np.nanquantile(d, 0.999), np.nanmax(d))
    assert np.quantile(d, 0.999) < 1e-4 and np.max(d) < 1e-3, (np.quantile(d, 0.999), np.max(d))
