"""Run-time compilation of the fit (Sec. 5).

CPU: NVRTC compiles the fit for both modes without a device, and the on-disk
cache serves a second build of the same variant without compiling.
GPU: the kernel compiled at run time gives the ahead-of-time kernel's bits in
deterministic mode, stays within the fast-mode tolerance, and serves recorded
fits (the adjoint follows it) and batched frames."""
import numpy as np
import pytest

from paper_2511_17018_gb300 import synth
from paper_2511_17018_gb300 import tpcfit as tf


def _need_nvrtc():
    if not tf.tpcfit_rtc_available():
        pytest.skip("NVRTC not available")


def test_rtc_builds_both_modes_and_caches_on_disk(tmp_path):
    _need_nvrtc()
    g = synth.default_geometry()
    d = str(tmp_path)
    n0 = tf.tpcfit_rtc_compile_count()
    tf.tpcfit_rtc_build(g, 0.5, False, 4, 24, cache_dir=d)
    tf.tpcfit_rtc_build(g, 0.5, True, 4, 24, record=True, cache_dir=d)
    assert tf.tpcfit_rtc_compile_count() == n0 + 2
    files = sorted(p.name for p in tmp_path.iterdir())
    assert len([f for f in files if f.endswith(".cubin")]) == 2 and len(files) == 4
    tf.tpcfit_rtc_build(g, 0.5, False, 4, 24, cache_dir=d)        # served from disk
    assert tf.tpcfit_rtc_compile_count() == n0 + 2
    tf.tpcfit_rtc_build(g, 0.4, False, 4, 24, cache_dir=d)        # another field: another kernel
    assert tf.tpcfit_rtc_compile_count() == n0 + 3


def test_rtc_build_rejects_bad_shape():
    _need_nvrtc()
    with pytest.raises(tf.TpcfitError) as e:
        tf.tpcfit_rtc_build(synth.default_geometry(), 0.5, False, 4, 7)
    assert e.value.status == tf.EINVAL


torch = pytest.importorskip("torch")


def _host(out):
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _bits_equal(a, b):
    return all(np.array_equal(np.ascontiguousarray(a[k]).view(np.int32), np.ascontiguousarray(b[k]).view(np.int32))
               for k in ("params", "cov", "chi2", "ndf"))


@pytest.mark.gpu
@pytest.mark.parametrize("det", [True, False])
def test_rtc_fit_matches_ahead_of_time_fit(det):
    _need_nvrtc()
    import oracle
    from paper_2511_17018_gb300 import tolerance
    fr = synth.generate(20000, 2, drop_p=0.05, cap_lengths=True)
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz, deterministic=det)
    try:
        aot = _host(f.fit(dev))
        f.set_rtc(True)
        for rps, warps in ((4, 24), (8, 16)):
            f.set_config(1, rps, warps, True)
            rtc = _host(f.fit(dev))
            if det:
                assert _bits_equal(rtc, aot), (rps, warps)
            else:
                rep = tolerance.compare_to_fp64(rtc, oracle.fit(fr, "f64"))
                assert rep["ok"], rep
        assert f.status()[0] == tf.OK
    finally:
        f.close()


@pytest.mark.gpu
def test_rtc_recorded_fit_feeds_the_adjoint():
    _need_nvrtc()
    d_true = synth.alignment_offsets(3)
    fr = synth.generate(3000, 3, drop_p=0.05, cap_lengths=True, d_true=d_true)
    dev = tf.frame_to_device(fr)
    w = torch.ones(fr.n_tracks, device="cuda")
    grads = []
    for rtc in (False, True):
        f = tf.Fitter(fr.geometry, fr.bz, deterministic=True)
        try:
            f.set_alignment(torch.from_numpy(d_true).cuda())
            f.set_rtc(rtc)
            f.set_record(True)
            out = f.fit(dev)
            ga, gs = f.backward(dev, out, w)
            torch.cuda.synchronize()
            grads.append((ga.cpu().numpy(), gs.cpu().numpy()))
        finally:
            f.close()
    for a, b in zip(grads[0], grads[1]):
        assert np.array_equal(a.view(np.int32), b.view(np.int32))


@pytest.mark.gpu
def test_rtc_batched_frames_and_disk_cache(tmp_path):
    _need_nvrtc()
    from paper_2511_17018_gb300.frames import FrameBatch, fit_frames
    frames = [synth.generate(n, 10 + i, drop_p=0.05, cap_lengths=True) for i, n in enumerate((700, 1500, 300))]
    batch = FrameBatch.from_frames(frames)
    outs = []
    for rtc in (False, True):
        f = tf.Fitter(frames[0].geometry, frames[0].bz, deterministic=True)
        try:
            f.set_rtc(rtc, str(tmp_path) if rtc else None)
            outs.append(_host(fit_frames(f, batch)))
        finally:
            f.close()
    assert _bits_equal(outs[0], outs[1])
    assert any(p.suffix == ".cubin" for p in tmp_path.iterdir())
    n = tf.tpcfit_rtc_compile_count()
    f = tf.Fitter(frames[0].geometry, frames[0].bz, deterministic=True)
    try:
        f.set_rtc(True, str(tmp_path))
        _host(fit_frames(f, batch))      # the same variant: memory or disk, no compilation
        assert tf.tpcfit_rtc_compile_count() == n
    finally:
        f.close()
