"""Alignment recovery (fit + adjoint + Adam)."""
import numpy as np
import pytest

from paper_2511_17018_gb300 import synth


def test_weak_mode_projection_removes_exactly_the_weak_modes():
    from paper_2511_17018_gb300 import align
    g = synth.default_geometry()
    rng = np.random.default_rng(1)
    X = g.row_x
    weak = np.zeros((36, 152, 2))
    for s in range(36):
        a, b, c = rng.normal(size=3)
        weak[s, :, 0] = a + b * X + c * X ** 2
        a, b = rng.normal(size=2)
        weak[s, :, 1] = a + b * X
    raw, proj = align.recovery(weak, np.zeros_like(weak), X)
    assert raw > 0.1 and proj < 1e-9
    noise = rng.normal(0, 0.05, (36, 152, 2))
    raw, proj = align.recovery(noise, np.zeros_like(noise), X)
    assert abs(proj / raw - np.sqrt(1 - 5 / 304)) < 0.05  # 5 of 304 directions per sector removed


@pytest.mark.gpu
def test_alignment_loop_recovers_offsets():
    torch = pytest.importorskip("torch")
    from paper_2511_17018_gb300 import align
    from paper_2511_17018_gb300 import tpcfit as tf
    d_true = synth.alignment_offsets(5)
    fr = synth.generate(40000, 55, drop_p=0.05, cap_lengths=True, d_true=d_true)
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        loop = align.AlignmentLoop(f, dev, lr=5e-3)
        losses = loop.run(40)
        d_est = loop.d.cpu().numpy()
        raw0, proj0 = align.recovery(np.zeros_like(d_true), d_true, fr.geometry.row_x)
        raw, proj = align.recovery(d_est, d_true, fr.geometry.row_x)
        assert losses[-1] < 0.9 * losses[0]
        assert proj < 0.5 * proj0, (proj0, proj, raw0, raw)
        # the graph replay matches an eager iteration from the same state
        eager = align.AlignmentLoop(f, dev, lr=5e-3, use_graph=False)
        l2 = eager.run(3)
        loop.reset()
        l1 = loop.run(3)
        assert np.allclose(l1, l2, rtol=1e-5)
    finally:
        f.close()
