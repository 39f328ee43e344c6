"""Autotuner host logic (CPU) and its effect on results (GPU)."""
import numpy as np
import pytest

from paper_2511_17018_gb300 import synth


def test_cache_roundtrip(tmp_path):
    from paper_2511_17018_gb300 import autotune
    p = str(tmp_path / "at.json")
    assert autotune.load_cache(p) == {}
    autotune.save_cache({"k": {"rows_per_stage": 4}}, p)
    assert autotune.load_cache(p) == {"k": {"rows_per_stage": 4}}


def test_candidates_cover_the_documented_sweep():
    from paper_2511_17018_gb300 import autotune
    c = list(autotune.candidates())
    assert {x[0] for x in c} == {1, 2, 4, 8, 16, 32}   # tracks per warp 32, 16, 8, 4, 2, 1
    assert {x[1] for x in c} == {4, 8, 16}
    assert len(c) == len(set(c))


def test_sample_keeps_the_length_histogram():
    from paper_2511_17018_gb300 import autotune
    fr = synth.generate(30000, 2, drop_p=0.05, cap_lengths=True)
    idx = autotune.sample_tracks(fr, fraction=0.01, minimum=5000)
    assert len(idx) == 5000 and np.all(np.diff(idx) > 0)
    a = np.histogram(fr.lengths(), bins=10, range=(0, 160))[0] / fr.n_tracks
    b = np.histogram(fr.lengths()[idx], bins=10, range=(0, 160))[0] / len(idx)
    assert np.abs(a - b).max() < 0.02


@pytest.mark.gpu
def test_tuned_configuration_gives_identical_deterministic_results(tmp_path):
    torch = pytest.importorskip("torch")
    from paper_2511_17018_gb300 import autotune
    from paper_2511_17018_gb300 import tpcfit as tf
    fr = synth.generate(20000, 2, drop_p=0.05, cap_lengths=True)
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz, deterministic=True)
    try:
        base = {k: v.cpu().numpy() for k, v in f.fit(dev).items()}
        best = autotune.tune(f, dev, fr.lengths(), mode="det", reps=2, cache_path=str(tmp_path / "c.json"))
        assert best["tried"] >= 6 and best["ms"] > 0
        got = {k: v.cpu().numpy() for k, v in f.fit(dev).items()}
        for k in base:
            assert np.array_equal(base[k].view(np.int32), got[k].view(np.int32))
        again = autotune.tune(f, dev, fr.lengths(), mode="det", cache_path=str(tmp_path / "c.json"))
        assert again["key"] == best["key"]   # served from the cache
    finally:
        f.close()
