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


def _bare_loop(n=10, lr=5e-3):
    """An AlignmentLoop's state without a fitter (CPU tensors), for the file logic."""
    torch = pytest.importorskip("torch")
    from paper_2511_17018_gb300 import align
    lp = align.AlignmentLoop.__new__(align.AlignmentLoop)
    lp.n, lp.lr, lp.b1, lp.b2, lp.eps = n, lr, 0.9, 0.999, 1e-8
    lp.d = torch.zeros(36 * 152 * 2)
    lp.m = torch.zeros_like(lp.d)
    lp.v = torch.zeros_like(lp.d)
    lp.t = torch.zeros(())
    return lp


def test_checkpoint_round_trip_and_checks(tmp_path):
    torch = pytest.importorskip("torch")
    a = _bare_loop()
    g = torch.Generator().manual_seed(3)
    for x in (a.d, a.m, a.v):
        x.copy_(torch.randn(x.shape, generator=g))
    a.t.fill_(17.0)
    path = str(tmp_path / "loop.pt")
    a.save(path)
    a.save(path)  # replaced in place
    assert sorted(p.name for p in tmp_path.iterdir()) == ["loop.pt"]  # no temporary left behind
    b = _bare_loop()
    b.load(path)
    for k in ("d", "m", "v", "t"):
        assert torch.equal(getattr(a, k), getattr(b, k)), k
    assert b.iteration == 17
    with pytest.raises(ValueError):
        _bare_loop(lr=1e-3).load(path)
    with pytest.raises(ValueError):
        _bare_loop(n=11).load(path)


@pytest.mark.gpu
def test_alignment_loop_resumes_bit_for_bit(tmp_path):
    # deterministic mode: 3 iterations, checkpoint, 3 more; a fresh loop that
    # reads the checkpoint and runs 3 iterations ends on the same offsets
    torch = pytest.importorskip("torch")
    from paper_2511_17018_gb300 import align
    from paper_2511_17018_gb300 import tpcfit as tf
    d_true = synth.alignment_offsets(5)
    fr = synth.generate(6000, 56, drop_p=0.05, cap_lengths=True, d_true=d_true)
    dev = tf.frame_to_device(fr)
    path = str(tmp_path / "loop.pt")
    f = tf.Fitter(fr.geometry, fr.bz, deterministic=True)
    try:
        loop = align.AlignmentLoop(f, dev, lr=5e-3)
        loop.run(3, checkpoint=path, every=3)
        tail = loop.run(3)
        d_whole = loop.d.cpu().numpy()
    finally:
        f.close()
    f = tf.Fitter(fr.geometry, fr.bz, deterministic=True)
    try:
        again = align.AlignmentLoop(f, dev, lr=5e-3)
        again.load(path)
        assert again.iteration == 3
        tail2 = again.run(3)
        d_resumed = again.d.cpu().numpy()
    finally:
        f.close()
    assert np.array_equal(tail.view(np.int32), tail2.view(np.int32))
    assert np.array_equal(d_whole.view(np.int32), d_resumed.view(np.int32))
    assert np.abs(d_whole).max() > 0
