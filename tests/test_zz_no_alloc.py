"""tpcfit_fit_noalloc, the entry point for callers that cannot allocate device
memory (for example code inside someone else's stream capture or an
allocation-free real-time loop), against tpcfit_fit.

It keeps its scratch in a static device array, so two calls in a row must not
see each other's leftovers; the file is named to run last so that a failure
here cannot hide the other GPU tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_17018_gb300 import synth, tolerance  # noqa: E402
from paper_2511_17018_gb300 import tpcfit as tf  # noqa: E402


def _run_noalloc(fr, deterministic, align=None):
    dev = tf.frame_to_device(fr)
    out = tf.empty_outputs(fr.n_tracks)
    out["params"].fill_(7.0)  # stale values must be overwritten
    tf.tpcfit_fit_noalloc(fr.geometry, fr.bz, align, deterministic, dev["y"], dev["z"], dev["rowsec"],
                          dev["offsets"], dev["seeds"], out["params"], out["cov"], out["chi2"], out["ndf"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _run_handle(fr, deterministic, align=None):
    f = tf.Fitter(fr.geometry, fr.bz, deterministic=deterministic)
    try:
        if align is not None:
            f.set_alignment(align)
        out = f.fit(tf.frame_to_device(fr))
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        f.close()


def _same_bits(a, b):
    return all(np.array_equal(np.ascontiguousarray(a[k]).view(np.int32), np.ascontiguousarray(b[k]).view(np.int32))
               for k in ("params", "cov", "chi2", "ndf"))


def test_noalloc_matches_fit_on_two_calls_in_a_row():
    a = synth.generate(20000, 41, drop_p=0.05, cap_lengths=True)
    b = synth.generate(7000, 42, drop_p=0.05, cap_lengths=True, d_true=synth.alignment_offsets(42))
    d = torch.from_numpy(b.d_true).cuda()
    for det in (True, False):
        first = _run_noalloc(a, det)
        second = _run_noalloc(b, det, align=d)
        ref_a = _run_handle(a, det)
        ref_b = _run_handle(b, det, align=d)
        if det:
            assert _same_bits(first, ref_a)
            assert _same_bits(second, ref_b)
        else:
            for got, ref in ((first, ref_a), (second, ref_b)):
                assert np.array_equal(got["ndf"], ref["ndf"])
                rep = tolerance.compare_to_fp64(got, {k: v.astype(np.float64) if v.dtype == np.float32 else v
                                                      for k, v in ref.items()})
                assert rep["ok"], rep


def test_noalloc_rejects_sizes_beyond_its_scratch():
    fr = synth.generate(10, 43)
    dev = tf.frame_to_device(fr)
    out = tf.empty_outputs(10)
    big = torch.zeros(tf.NOALLOC_MAX_TRACKS + 2, dtype=torch.int32, device="cuda")
    seeds = torch.zeros((5, tf.NOALLOC_MAX_TRACKS + 1), dtype=torch.float32, device="cuda")
    with pytest.raises(tf.TpcfitError) as e:
        tf.tpcfit_fit_noalloc(fr.geometry, fr.bz, None, 0, dev["y"], dev["z"], dev["rowsec"], big, seeds,
                              torch.empty((5, tf.NOALLOC_MAX_TRACKS + 1), device="cuda"),
                              torch.empty((15, tf.NOALLOC_MAX_TRACKS + 1), device="cuda"),
                              torch.empty(tf.NOALLOC_MAX_TRACKS + 1, device="cuda"),
                              torch.empty(tf.NOALLOC_MAX_TRACKS + 1, dtype=torch.int32, device="cuda"))
    assert e.value.status == tf.EINVAL


def test_noalloc_bad_track_is_flagged_and_the_next_call_is_clean():
    # one track with a row beyond the geometry: that track alone gets ndf = -2
    # and NaNs; a clean call afterwards equals tpcfit_fit bit for bit, so the
    # shared array's error word and work counter carry nothing over
    fr = synth.generate(3000, 44, drop_p=0.05, cap_lengths=True)
    bad = fr.subset(np.arange(fr.n_tracks))
    bad.rowsec = bad.rowsec.copy()
    t = 1234
    bad.rowsec[bad.offsets[t] + 2] = np.uint16((160 << 6) | (int(bad.rowsec[bad.offsets[t] + 2]) & 63))
    got = _run_noalloc(bad, True)
    ref = _run_handle(fr, True)
    assert got["ndf"][t] == -2
    assert np.all(np.isnan(got["params"][:, t])) and np.isnan(got["chi2"][t])
    keep = np.arange(fr.n_tracks) != t
    for k in ("params", "cov", "chi2", "ndf"):
        a = np.ascontiguousarray(got[k][..., keep]).view(np.int32)
        b = np.ascontiguousarray(ref[k][..., keep]).view(np.int32)
        assert np.array_equal(a, b), k
    assert _same_bits(_run_noalloc(fr, True), ref)
