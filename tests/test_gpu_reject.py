"""Outlier rejection after the smoother (run on a GB300 with -m gpu).

The selection is integer work: the kept clusters and the new offsets must
equal, element for element, a plain numpy selection of the same chi2 values
(NaN kept, cut exclusive).  On tracks with one cluster displaced by 10 sigma,
the smoother's chi2 with a 2-dof cut finds the displaced clusters, and the
refit of what is kept has the chi2 / ndf of clean tracks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_17018_gb300 import synth  # noqa: E402
from paper_2511_17018_gb300 import tpcfit as tf  # noqa: E402


def _numpy_reject(fr, chi2, cut):
    keep = ~(chi2 > cut)
    lens = np.add.reduceat(keep.astype(np.int64), fr.offsets[:-1]) if fr.n_hits else np.zeros(fr.n_tracks, np.int64)
    lens[np.diff(fr.offsets) == 0] = 0
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    return fr.y[keep], fr.z[keep], fr.rowsec[keep], off


@pytest.mark.parametrize("cut", [0.0, 2.0, 9.0, 1e30])
def test_selection_equals_numpy(cut):
    fr = synth.generate(3000, 41, drop_p=0.05, cap_lengths=True)
    rng = np.random.default_rng(3)
    chi2 = rng.exponential(2.0, fr.n_hits).astype(np.float32)
    chi2[rng.random(fr.n_hits) < 0.01] = np.nan
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        got = f.reject_outliers(dev, torch.from_numpy(chi2).cuda(), cut)
        torch.cuda.synchronize()
    finally:
        f.close()
    y, z, rs, off = _numpy_reject(fr, chi2, cut)
    assert np.array_equal(got["offsets"].cpu().numpy(), off)
    assert np.array_equal(got["y"].cpu().numpy().view(np.int32), y.view(np.int32))
    assert np.array_equal(got["z"].cpu().numpy().view(np.int32), z.view(np.int32))
    assert np.array_equal(got["rowsec"].cpu().numpy().view(np.uint16), rs)


def test_edge_cases():
    fr = synth.generate(50, 42)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        # no tracks
        off = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        e = torch.empty(0, device="cuda")
        tf.tpcfit_reject_outliers(f.h, e, e, torch.empty(0, dtype=torch.int16, device="cuda"),
                                  torch.zeros(1, dtype=torch.int32, device="cuda"), e, 1.0, e, e,
                                  torch.empty(0, dtype=torch.int16, device="cuda"), off)
        torch.cuda.synchronize()
        assert int(off[0]) == 0
        # an empty track, and a last track whose offsets run backwards, keep
        # nothing (no two ranges overlap)
        dev = tf.frame_to_device(fr)
        offsets = dev["offsets"].clone()
        n = fr.n_tracks
        offsets[10] = offsets[9]                # track 9 empty; track 10 takes its clusters
        offsets[n] = offsets[n - 1] - 1         # the last track runs backwards
        chi2 = torch.zeros(fr.n_hits, device="cuda")
        d2 = dict(dev, offsets=offsets)
        got = f.reject_outliers(d2, chi2, 1.0)
        o = got["offsets"].cpu().numpy()
        lens = np.diff(o)
        assert lens[9] == 0 and lens[n - 1] == 0
        assert lens[10] == fr.offsets[11] - fr.offsets[9]
        assert o[-1] == fr.offsets[n - 1]
        with pytest.raises(tf.TpcfitError) as err:
            f.reject_outliers(dev, chi2, float("nan"))
        assert err.value.status == tf.EINVAL
        with pytest.raises(tf.TpcfitError):
            f.reject_outliers(dev, chi2, -1.0)
    finally:
        f.close()


def test_displaced_clusters_are_rejected_and_the_refit_is_clean():
    fr = synth.generate(4000, 31, drop_p=0.05, cap_lengths=True)
    off = fr.offsets
    moved = off[:-1] + np.diff(off) // 2
    fr.y = fr.y.copy()
    fr.y[moved] += np.float32(1.0)             # 10 sigma
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        f.set_record(True)
        out = f.fit(dev)
        sm = f.smooth(dev, out)
        chi2 = sm["chi2"]
        cut = 16.0                             # 2-dof tail probability 3.4e-4
        clean = f.reject_outliers(dev, chi2, cut)
        f.set_record(False)
        out2 = f.fit(clean)
        torch.cuda.synchronize()
        c = chi2.cpu().numpy()
        ndf0 = out["ndf"].cpu().numpy()
        chi2b, ndfb = out2["chi2"].cpu().numpy(), out2["ndf"].cpu().numpy()
    finally:
        f.close()
    ok = ndf0 > 0
    dropped = c > cut
    hit_moved = np.zeros(fr.n_hits, bool)
    hit_moved[moved] = True
    # the displaced clusters of fitted tracks are found, and few clean ones are lost
    assert dropped[moved[ok]].mean() > 0.99
    assert dropped[~hit_moved & np.repeat(ok, np.diff(off))].mean() < 2e-3
    # the refit of the kept clusters: chi2 / ndf of clean tracks
    good = ndfb > 0
    assert good.mean() > 0.99
    assert abs(np.mean(chi2b[good] / ndfb[good]) - 1.0) < 0.05
