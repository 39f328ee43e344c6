"""Parity of the CUDA fit with the CPU oracle (run on a GB300 with -m gpu).

Fast mode: within the FP32-vs-FP64 tolerance of paper_2511_17018_gb300.tolerance.
Deterministic mode: bit-exact against the strict-FP32 oracle, run to run and
for every launch configuration."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2511_17018_gb300 import synth, tolerance  # noqa: E402
from paper_2511_17018_gb300 import tpcfit as tf  # noqa: E402


def _host(out):
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _bits_equal(a, b):
    for k in ("params", "cov", "chi2", "ndf"):
        x = np.ascontiguousarray(a[k]).view(np.int32)
        y = np.ascontiguousarray(b[k]).view(np.int32)
        if not np.array_equal(x, y):
            bad = np.nonzero(x != y)
            return f"{k}: {len(bad[0])} words differ, first at {tuple(i[0] for i in bad)}"
    return None


@pytest.fixture(scope="module")
def fitter():
    tf.load()
    f = tf.Fitter(synth.default_geometry(), 0.5)
    yield f
    f.close()


@pytest.fixture(scope="module")
def frames():
    return {
        "plain1000": synth.plain_frame(),
        "drop20k": synth.generate(20000, 2, drop_p=0.05, cap_lengths=True),
        "align5k": synth.generate(5000, 3, drop_p=0.05, cap_lengths=True, d_true=synth.alignment_offsets(3)),
    }


@pytest.mark.parametrize("name", ["plain1000", "drop20k"])
@pytest.mark.parametrize("form", [1, 0], ids=["ud", "sqrt"])
def test_fast_mode_matches_fp64_oracle(fitter, frames, name, form):
    # both factor forms of the fast fit (U-D, square root) against FP64
    fr = frames[name]
    fitter.set_mode(False)
    fitter.set_config(1, 4, 24, True)
    fitter.set_fit_form(form)
    try:
        got = _host(fitter.fit(tf.frame_to_device(fr)))
    finally:
        fitter.set_fit_form(1)
    ref = oracle.fit(fr, "f64")
    rep = tolerance.compare_to_fp64(got, ref)
    print(form, rep)
    assert rep["ok"], rep
    assert np.array_equal(got["ndf"], ref["ndf"])


@pytest.mark.parametrize("shape", [(4, 8), (4, 12), (8, 8), (8, 16), (16, 8)])
def test_fast_u_d_fit_in_every_shape(fitter, frames, shape):
    fr = frames["drop20k"]
    fitter.set_mode(False)
    try:
        fitter.set_config(1, shape[0], shape[1], shape[0] != 8)
        got = _host(fitter.fit(tf.frame_to_device(fr)))
    finally:
        fitter.set_config(1, 4, 24, True)
    rep = tolerance.compare_to_fp64(got, oracle.fit(fr, "f64"))
    assert rep["ok"], (shape, rep)


@pytest.mark.parametrize("name", ["plain1000", "drop20k"])
def test_deterministic_mode_bit_exact_vs_strict_fp32(fitter, frames, name):
    fr = frames[name]
    fitter.set_mode(True)
    fitter.set_config(1, 4, 24, True)
    got = _host(fitter.fit(tf.frame_to_device(fr)))
    ref = oracle.fit(fr, "f32")
    assert _bits_equal(got, ref) is None, _bits_equal(got, ref)


def test_deterministic_mode_independent_of_launch_config_and_runs(fitter, frames):
    fr = frames["drop20k"]
    dev = tf.frame_to_device(fr)
    fitter.set_mode(True)
    base = None
    for rps, warps in ((4, 8), (4, 12), (4, 24), (8, 8), (8, 16), (16, 8)):
        for srt in (True, False):
            fitter.set_config(1, rps, warps, srt)
            for _ in range(2):
                got = _host(fitter.fit(dev))
                if base is None:
                    base = got
                assert _bits_equal(got, base) is None, (rps, warps, srt)
    fitter.set_config(1, 4, 24, True)


def test_alignment_offsets_are_subtracted(fitter, frames):
    fr = frames["align5k"]
    d = torch.from_numpy(fr.d_true).cuda()
    fitter.set_alignment(d)
    try:
        fitter.set_mode(True)
        got = _host(fitter.fit(tf.frame_to_device(fr)))
        ref = oracle.fit(fr, "f32", align=fr.d_true)
        assert _bits_equal(got, ref) is None
        fitter.set_mode(False)
        got = _host(fitter.fit(tf.frame_to_device(fr)))
        rep = tolerance.compare_to_fp64(got, oracle.fit(fr, "f64", align=fr.d_true))
        assert rep["ok"], rep
    finally:
        fitter.set_alignment(None)


def test_edge_cases(fitter):
    fr = synth.generate(64, 31, drop_p=0.05, cap_lengths=True)
    lens = fr.lengths().copy()
    lens[0] = 0   # empty track
    lens[1] = 1   # one cluster
    lens[2] = 2   # two clusters
    lens[3] = 3   # minimal fit
    idx = np.concatenate([np.arange(o, o + l) for o, l in zip(fr.offsets[:-1], lens)])
    fr.y, fr.z, fr.rowsec = fr.y[idx], fr.z[idx], fr.rowsec[idx]
    fr.offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    fr.seeds[2, 5] = 0.9995   # unusable seed
    fitter.set_mode(True)
    got = _host(fitter.fit(tf.frame_to_device(fr)))
    ref = oracle.fit(fr, "f32")
    assert list(got["ndf"][:4]) == [-1, -1, -1, 1]
    assert got["ndf"][5] == -1
    assert _bits_equal(got, ref) is None
    # empty frame
    empty = fr.subset(np.arange(0))
    dev = tf.frame_to_device(empty)
    out = tf.empty_outputs(0)
    tf.tpcfit_fit(fitter.h, dev["y"], dev["z"], dev["rowsec"], dev["offsets"], dev["seeds"], out["params"],
                  out["cov"], out["chi2"], out["ndf"])
    assert fitter.status()[0] == tf.OK


def test_invalid_input_is_flagged_not_fatal(fitter):
    fr = synth.generate(100, 32)
    rs = fr.rowsec.copy()
    bad_track = 7
    rs[fr.offsets[bad_track] + 3] = (200 << 6) | 5   # row 200 does not exist
    fr.rowsec = rs
    fitter.set_mode(False)
    got = _host(fitter.fit(tf.frame_to_device(fr)))
    assert got["ndf"][bad_track] == -2
    assert np.all(got["ndf"][np.arange(100) != bad_track] > 0)
    st, code, trk = fitter.status()
    assert st == tf.EDEVICE and code == 2 and trk == bad_track
    assert fitter.status()[0] == tf.OK   # the word was cleared
    # offsets past the end of the hit arrays
    dev = tf.frame_to_device(fr)
    dev["offsets"][-1] = int(fr.n_hits) + 5
    _host(fitter.fit(dev))
    st, code, trk = fitter.status()
    assert st == tf.EDEVICE and code == 1 and trk == fr.n_tracks - 1


def test_binding_rejects_mismatched_sizes(fitter):
    # the C entry points see only pointers; the binding checks every array's
    # size against the track and cluster counts before it calls them
    fr = synth.generate(50, 34)
    dev = tf.frame_to_device(fr)
    out = tf.empty_outputs(50)
    short = tf.empty_outputs(49)
    y, z, rs, off, seeds = dev["y"], dev["z"], dev["rowsec"], dev["offsets"], dev["seeds"]
    with pytest.raises(ValueError):
        tf.tpcfit_fit(fitter.h, y, z[:-1], rs, off, seeds, out["params"], out["cov"], out["chi2"], out["ndf"])
    with pytest.raises(ValueError):
        tf.tpcfit_fit(fitter.h, y, z, rs, off, seeds, out["params"], short["cov"], out["chi2"], out["ndf"])
    with pytest.raises(ValueError):
        tf.tpcfit_fit_noalloc(fr.geometry, fr.bz, None, 0, y, z, rs, off, seeds, out["params"], out["cov"],
                              short["chi2"], out["ndf"])
    base = torch.tensor([0, 50], dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        tf.tpcfit_fit_frames(fitter.h, y, z, rs, off, base, seeds[:, :49].contiguous(), out["params"], out["cov"],
                             out["chi2"], out["ndf"])
    with pytest.raises(ValueError):
        tf.tpcfit_fit_frames(fitter.h, y, z, rs, off, base, seeds, out["params"], out["cov"], out["chi2"],
                             out["ndf"], frame_ready=torch.zeros(2, dtype=torch.int32, device="cuda"))
    g = torch.zeros(50, device="cuda")
    with pytest.raises(ValueError):
        tf.tpcfit_fit_backward(fitter.h, y, z, rs, off, out["ndf"], g, torch.empty(36 * 152 * 2, device="cuda"),
                               torch.empty((5, 50), device="cuda"), grad_meas=torch.empty(y.numel(), device="cuda"))
    with pytest.raises(ValueError):
        tf.tpcfit_smooth(fitter.h, y, z, rs, off, short["ndf"], torch.empty((y.numel(), 2), device="cuda"),
                         torch.empty((y.numel(), 3), device="cuda"), torch.empty(y.numel(), device="cuda"))
    # nothing was enqueued: a correct call still works and the error word is clear
    tf.tpcfit_fit(fitter.h, y, z, rs, off, seeds, out["params"], out["cov"], out["chi2"], out["ndf"])
    assert np.all(_host(out)["ndf"] > 0)
    assert fitter.status()[0] == tf.OK


def test_host_buffer_entry_point_equals_device_entry_point(fitter, frames):
    fr = frames["drop20k"]
    fitter.set_mode(True)
    dev = _host(fitter.fit(tf.frame_to_device(fr)))
    host = tf.tpcfit_fit_host(fitter.h, fr.y, fr.z, fr.rowsec, fr.offsets, np.ascontiguousarray(fr.seeds))
    assert _bits_equal(dev, host) is None


def test_full_size_time_frame_sampled(fitter):
    # 400,000 tracks in one launch (the time-frame-sized batch); the oracle checks
    # a seeded sample of 3,000 tracks one by one
    fr = synth.time_frame()
    dev = tf.frame_to_device(fr)
    rng = np.random.default_rng(77)
    sample = np.sort(rng.choice(fr.n_tracks, 3000, replace=False))
    sub = fr.subset(sample)
    fitter.set_mode(False)
    got = _host(fitter.fit(dev))
    gs = {k: (v[:, sample] if v.ndim == 2 else v[sample]) for k, v in got.items()}
    rep = tolerance.compare_to_fp64(gs, oracle.fit(sub, "f64"))
    assert rep["ok"], rep
    assert np.all(got["ndf"] >= -1)
    fitter.set_mode(True)
    got = _host(fitter.fit(dev))
    gs = {k: (v[:, sample] if v.ndim == 2 else v[sample]) for k, v in got.items()}
    assert _bits_equal(gs, oracle.fit(sub, "f32")) is None
    assert fitter.status()[0] == tf.OK


@pytest.mark.parametrize("lanes", [2, 4, 8, 16, 32])
def test_lanes_per_track_variants(fitter, frames, lanes):
    # 32 / lanes tracks per warp: the factor's columns split over a track's
    # lanes, the column sums gathered in column order -- bit-identical to the
    # strict-FP32 reference in deterministic mode, within tolerance in fast mode
    fr = frames["drop20k"]
    dev = tf.frame_to_device(fr)
    try:
        fitter.set_config(lanes, 4, 24, True)
        fitter.set_mode(True)
        got = _host(fitter.fit(dev))
        assert _bits_equal(got, oracle.fit(fr, "f32")) is None
        fitter.set_mode(False)
        got = _host(fitter.fit(dev))
        rep = tolerance.compare_to_fp64(got, oracle.fit(fr, "f64"))
        assert rep["ok"], rep
    finally:
        fitter.set_config(1, 4, 24, True)


def test_lanes_per_track_shapes_and_fallbacks(fitter):
    # several lanes per track come in one shape; other shapes are refused
    for bad in ((2, 8, 16), (4, 4, 12), (3, 4, 24), (64, 4, 24)):
        with pytest.raises(tf.TpcfitError):
            fitter.set_config(bad[0], bad[1], bad[2], True)
    fitter.set_config(1, 4, 24, True)


def test_lanes_recording_feeds_the_same_adjoint():
    # a fit recorded with 8 lanes per track leaves the checkpoints the one-lane
    # fit leaves: the deterministic adjoint is bit for bit the same
    fr = synth.generate(3000, 9, drop_p=0.05, cap_lengths=True)
    dev = tf.frame_to_device(fr)
    g = torch.from_numpy(np.random.default_rng(2).uniform(0.5, 2, fr.n_tracks).astype(np.float32)).cuda()
    res = []
    for lanes in (1, 8, 2):
        f = tf.Fitter(fr.geometry, fr.bz, deterministic=True)
        try:
            f.set_config(lanes, 4, 24, True)
            f.set_record(True)
            out = f.fit(dev)
            gm = torch.empty((fr.n_hits, 2), device="cuda")
            ga, gs = f.backward(dev, out, g, gm)
            torch.cuda.synchronize()
            res.append([x.cpu().numpy().view(np.int32).copy() for x in (gm, ga, gs, out["chi2"])])
        finally:
            f.close()
    for other in res[1:]:
        for a, b in zip(res[0], other):
            assert np.array_equal(a, b)
