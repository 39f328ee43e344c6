"""Two-filter smoother on the GPU against the FP64 oracle (run on a GB300 with -m gpu).

Per cluster the leave-one-out residual, its covariance and chi2 agree with the
oracle's information-form combination within the FP32 tolerance below (the
same FP32-vs-FP64 rounding argument as for the fit: residuals of ~0.1 cm
carried through ~150 steps); the deterministic mode repeats bit for bit; a
displaced cluster is flagged."""
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
