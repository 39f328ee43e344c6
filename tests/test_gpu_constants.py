"""Per-time-frame constants travel with each launch (run on a GB300 with -m gpu).

Two handles with different constants (field, material) fitting on two streams
whose work overlaps must each reproduce their own strict-FP32 oracle bit for
bit, and a captured CUDA graph must replay with the constants it was captured
with, whatever other handles or the handle-free entry point ran in between."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2511_17018_gb300 import synth  # noqa: E402
from paper_2511_17018_gb300 import tpcfit as tf  # noqa: E402
from paper_2511_17018_gb300.frames import FrameBatch, GraphedFrameFit  # noqa: E402


def _bits(d):
    return {k: np.ascontiguousarray(v.cpu().numpy()).view(np.int32).copy() for k, v in d.items()}


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in ("params", "cov", "chi2", "ndf"))


def _oracle_bits(fr):
    r = oracle.fit(fr, "f32")
    return {k: np.ascontiguousarray(r[k]).view(np.int32) for k in ("params", "cov", "chi2", "ndf")}


def test_two_handles_with_different_constants_on_overlapping_streams():
    base = synth.generate(30000, 51, drop_p=0.05, cap_lengths=True)
    fa = base.subset(np.arange(base.n_tracks))           # Bz 0.5 T, no material
    fb = base.subset(np.arange(base.n_tracks))
    fb.bz = 0.42                                         # another field ...
    fb.material = synth.TPC_GAS                          # ... and the gas layers
    A = tf.Fitter(fa.geometry, fa.bz, deterministic=True)
    B = tf.Fitter(fb.geometry, fb.bz, deterministic=True)
    try:
        B.set_material(fb.material)
        dev = tf.frame_to_device(base)
        sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
        sa.wait_stream(torch.cuda.current_stream())
        sb.wait_stream(torch.cuda.current_stream())
        outs = []
        for _ in range(3):   # interleaved, nothing waits in between
            oa = tf.empty_outputs(base.n_tracks)
            ob = tf.empty_outputs(base.n_tracks)
            with torch.cuda.stream(sa):
                A.fit(dev, oa, stream=sa)
            with torch.cuda.stream(sb):
                B.fit(dev, ob, stream=sb)
            outs.append((oa, ob))
        torch.cuda.synchronize()
        want_a, want_b = _oracle_bits(fa), _oracle_bits(fb)
        assert not _same(want_a, want_b)
        for oa, ob in outs:
            assert _same(_bits(oa), want_a)
            assert _same(_bits(ob), want_b)
    finally:
        A.close()
        B.close()


def test_graph_replay_keeps_the_constants_it_was_captured_with():
    frames = [synth.generate(n, 60 + i, drop_p=0.05, cap_lengths=True) for i, n in enumerate((3000, 1200, 5000))]
    batch = FrameBatch.from_frames(frames)
    cat = synth.concat(frames)
    f = tf.Fitter(cat.geometry, cat.bz, deterministic=True)
    other = tf.Fitter(cat.geometry, 0.3, deterministic=True)
    try:
        g = GraphedFrameFit(f, batch)
        first = _bits(g.replay())
        torch.cuda.synchronize()
        # other constants in between: another handle, the handle-free entry point
        dev = tf.frame_to_device(cat)
        other.set_field(synth.FieldMap(0.3, -0.2))
        other.fit(dev)
        out = tf.empty_outputs(cat.n_tracks)
        tf.tpcfit_fit_noalloc(cat.geometry, 0.35, None, 1, dev["y"], dev["z"], dev["rowsec"], dev["offsets"],
                              dev["seeds"], out["params"], out["cov"], out["chi2"], out["ndf"])
        again = _bits(g.replay())
        torch.cuda.synchronize()
        assert _same(first, again)
        assert _same(first, _oracle_bits(cat))
    finally:
        f.close()
        other.close()
