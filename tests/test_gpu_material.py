"""Material layers at the pad rows and the field map on the GPU (run on a
GB300 with -m gpu).

Deterministic mode: bit-exact against the strict-FP32 oracle with material
(energy loss and the square-root noise folding in their canonical order) and
with the field map (midpoint curvature); fast mode within the FP32 tolerance
of the FP64 oracle; the smoother, the batched-frame and run-time-compiled fits
follow both; so does the adjoint (against the oracle's FP64 forward-mode
gradient)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2511_17018_gb300 import synth, tolerance  # noqa: E402
from paper_2511_17018_gb300 import tpcfit as tf  # noqa: E402

THICK = synth.Material(300.0, 2e-4)


def _host(out):
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _bits_equal(a, b):
    return all(np.array_equal(np.ascontiguousarray(a[k]).view(np.int32), np.ascontiguousarray(b[k]).view(np.int32))
               for k in ("params", "cov", "chi2", "ndf"))


@pytest.fixture(scope="module")
def frame():
    return synth.generate(8000, 12, drop_p=0.05, cap_lengths=True)


@pytest.mark.parametrize("mat", [synth.TPC_GAS, THICK], ids=["gas", "thick"])
def test_deterministic_fit_with_material_bit_exact(frame, mat):
    fr = frame.subset(np.arange(frame.n_tracks))
    fr.material = mat
    ref = oracle.fit(fr, "f32")
    f = tf.Fitter(fr.geometry, fr.bz, deterministic=True)
    try:
        f.set_material(mat)
        dev = tf.frame_to_device(fr)
        for rps, warps, srt in ((4, 24, True), (4, 12, False), (8, 16, True)):
            f.set_config(1, rps, warps, srt)
            assert _bits_equal(_host(f.fit(dev)), ref), (rps, warps, srt)
    finally:
        f.close()


@pytest.mark.parametrize("mat", [synth.TPC_GAS, THICK], ids=["gas", "thick"])
def test_fast_fit_with_material_within_tolerance(frame, mat):
    fr = frame.subset(np.arange(frame.n_tracks))
    fr.material = mat
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        f.set_material(mat)
        got = _host(f.fit(tf.frame_to_device(fr)))
    finally:
        f.close()
    rep = tolerance.compare_to_fp64(got, oracle.fit(fr, "f64"))
    assert rep["ok"], rep


def test_material_off_again_restores_the_plain_fit(frame):
    dev = tf.frame_to_device(frame)
    f = tf.Fitter(frame.geometry, frame.bz, deterministic=True)
    try:
        base = _host(f.fit(dev))
        f.set_material(THICK)
        with_mat = _host(f.fit(dev))
        f.set_material(None)
        again = _host(f.fit(dev))
    finally:
        f.close()
    assert _bits_equal(base, again)
    assert not _bits_equal(base, with_mat)


def test_smoother_with_material_matches_oracle(frame):
    from test_gpu_smooth import compare
    fr = frame.subset(np.arange(frame.n_tracks))
    fr.material = THICK
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        f.set_material(THICK)
        f.set_record(True)
        out = f.fit(dev)
        got = _host(f.smooth(dev, out))
    finally:
        f.close()
    rep = compare(got, oracle.smooth(fr))
    assert rep["nan_agree"] > 0.9999, rep
    assert rep["resid_ok"] > 0.999 and rep["rcov_ok"] > 0.999 and rep["chi2_ok"] > 0.999, rep


def test_batched_frames_and_run_time_compiled_fit_with_material(frame):
    from paper_2511_17018_gb300.frames import FrameBatch, fit_frames
    parts = [frame.subset(np.arange(a, b)) for a, b in ((0, 3000), (3000, 3500), (3500, 8000))]
    f = tf.Fitter(frame.geometry, frame.bz, deterministic=True)
    try:
        f.set_material(THICK)
        dev = tf.frame_to_device(frame)
        ref = _host(f.fit(dev))
        got = _host(fit_frames(f, FrameBatch.from_frames(parts)))
        assert _bits_equal(got, ref)
        if tf.tpcfit_rtc_available():
            f.set_rtc(True)
            assert _bits_equal(_host(f.fit(dev)), ref)
    finally:
        f.close()


FIELD = synth.FieldMap(0.3, -0.2)


@pytest.mark.parametrize("with_mat", [False, True], ids=["field", "field+gas"])
def test_field_map_fit_parity(frame, with_mat):
    # (the thick layers stop the 0.2 GeV/c tracks of this frame within a few
    # rows, where FP32 and FP64 may part at the stopping row; the gas does not)
    fr = frame.subset(np.arange(frame.n_tracks))
    fr.field = FIELD
    fr.material = synth.TPC_GAS if with_mat else None
    ref32, ref64 = oracle.fit(fr, "f32"), oracle.fit(fr, "f64")
    for det in (True, False):
        f = tf.Fitter(fr.geometry, fr.bz, deterministic=det)
        try:
            f.set_field(FIELD)
            f.set_material(fr.material)
            got = _host(f.fit(tf.frame_to_device(fr)))
        finally:
            f.close()
        if det:
            assert _bits_equal(got, ref32)
        else:
            rep = tolerance.compare_to_fp64(got, ref64)
            assert rep["ok"], {k: v for k, v in rep.items() if k != "worst"}


def test_field_map_smoother_frames_rtc_and_adjoint(frame):
    from test_gpu_smooth import compare
    from paper_2511_17018_gb300.frames import FrameBatch, fit_frames
    fr = frame.subset(np.arange(frame.n_tracks))
    fr.field = FIELD
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz, deterministic=True)
    try:
        f.set_field(FIELD)
        f.set_record(True)
        out = f.fit(dev)
        ref = _host(out)
        sm = _host(f.smooth(dev, out))
        f.set_record(False)
        parts = [fr.subset(np.arange(a, b)) for a, b in ((0, 5000), (5000, 8000))]
        assert _bits_equal(_host(fit_frames(f, FrameBatch.from_frames(parts))), ref)
        if tf.tpcfit_rtc_available():
            f.set_rtc(True)
            assert _bits_equal(_host(f.fit(dev)), ref)
        f.set_rtc(False)
        f.set_field(None)
        assert not _bits_equal(_host(f.fit(dev)), ref)
    finally:
        f.close()
    rep = compare(sm, oracle.smooth(fr))
    assert rep["nan_agree"] > 0.9999, rep
    assert rep["resid_ok"] > 0.999 and rep["rcov_ok"] > 0.999 and rep["chi2_ok"] > 0.999, rep


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


PHYS = {"field": (FIELD, None), "gas": (None, synth.TPC_GAS), "thick": (None, THICK),
        "field+gas": (FIELD, synth.TPC_GAS)}


def _thick_frame(n, seed):
    """Tracks of 1-5 GeV/c through the thick layers, simulated with their
    scattering and energy loss (sector 0).  On the slow tracks of the generic
    frame the thick layers make a few chi2 values extremely sensitive to their
    clusters (derivatives of ~1e4 per cm), beyond what an FP32 gradient can
    follow; these tracks are not."""
    rng = np.random.default_rng(seed)
    qpt = rng.choice([-1, 1], n) / rng.uniform(1.0, 5.0, n)
    tanl = rng.uniform(-0.5, 0.5, n)
    phi0 = np.full(n, 0.5 * np.pi / 9) + rng.uniform(-0.03, 0.03, n)
    z0 = rng.normal(0, 5, n)
    return synth.simulate_material(qpt, tanl, phi0, z0, synth.default_geometry(), 0.5, THICK, rng=rng)


@pytest.mark.parametrize("phys", list(PHYS))
@pytest.mark.parametrize("det", [False, True], ids=["fast", "det"])
def test_adjoint_with_field_map_and_material_matches_forward_mode_oracle(frame, det, phys):
    # the reverse runs through the midpoint curvature (which moves with the
    # state and, in residual coordinates, with the previous cluster) and through
    # the layers (energy loss, and the noise folded into the factor); bounds as
    # in the uniform-field adjoint test.  Thick layers stop some of the slow
    # tracks, and FP32 and FP64 may stop them one row apart: those few tracks
    # are left out of the comparison (the thick case runs on fast tracks, see
    # _thick_frame).
    field, mat = PHYS[phys]
    fr = _thick_frame(1200, 21) if phys == "thick" else frame.subset(np.arange(2500))
    fr.field, fr.material = field, mat
    d = synth.alignment_offsets(3)
    w = np.random.default_rng(6).uniform(0.5, 2.0, fr.n_tracks).astype(np.float32)
    ref = oracle.grad(fr, weights=w.astype(np.float64), align=d)
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz, deterministic=det)
    try:
        f.set_field(field)
        f.set_material(mat)
        f.set_alignment(torch.from_numpy(d).cuda())
        f.set_record(True)
        out = f.fit(dev)
        gm = torch.empty((fr.n_hits, 2), device="cuda")
        ga, gs = f.backward(dev, out, torch.from_numpy(w).cuda(), gm)
        torch.cuda.synchronize()
        gm, ga, gs = gm.cpu().numpy(), ga.cpu().numpy(), gs.cpu().numpy()
        ndf = out["ndf"].cpu().numpy()
        if det:  # and run to run
            gm2 = torch.empty((fr.n_hits, 2), device="cuda")
            ga2, _ = f.backward(dev, out, torch.from_numpy(w).cuda(), gm2)
            assert np.array_equal(ga2.cpu().numpy().view(np.int32), ga.view(np.int32))
            assert np.array_equal(gm2.cpu().numpy().view(np.int32), gm.view(np.int32))
    finally:
        f.close()
    ok = ndf == ref["ndf"]
    assert ok.mean() > (0.999 if phys == "thick" else 1.0 - 1e-12), ok.mean()
    hit_ok = np.repeat(ok, np.diff(fr.offsets))
    assert _rel(gm[hit_ok], ref["grad_meas"][hit_ok]) < 5e-4
    assert _rel(gs[:, ok], ref["grad_seed"][:, ok]) < 5e-3
    # the alignment gradient is the per-key sum of the cluster gradients
    assert _rel(ga, oracle.align_grad_from_meas(fr, gm)) < 1e-5
    if ok.all():
        assert _rel(ga, oracle.align_grad_from_meas(fr, ref["grad_meas"])) < 5e-4
    if det:
        # against the exact gradient of the strict-FP32 sequence through the same
        # physics: only the reverse sweep's own rounding remains, also on the
        # slow thick-layer tracks whose gradient the FP32 forward cannot follow
        r32 = oracle.grad(fr, weights=w.astype(np.float64), align=d, precision="f32")
        assert np.array_equal(ndf, r32["ndf"])
        # (measured: 0.5-4e-6 in norm, 99.9% of elements within 8e-5; the
        # reverse of the material folding goes through the triangular inverse
        # of the folded factor, which costs accuracy on its worst elements)
        e = tolerance.gradient_errors(gm, r32["grad_meas"])
        assert e["norm"] <= 2e-5 and e["q999"] <= 3e-4 and e["max"] <= 0.1, e
    # without the physics the reverse would be far off
    bare = fr.subset(np.arange(fr.n_tracks))
    bare.field, bare.material = None, None
    ref0 = oracle.grad(bare, weights=w.astype(np.float64), align=d)
    assert _rel(ref0["grad_meas"][hit_ok], ref["grad_meas"][hit_ok]) > 1e-3
