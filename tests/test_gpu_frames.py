"""Batched time frames in one persistent launch (tpcfit_fit_frames), CUDA-graph
replay and frame-ready flags with bounded waits (run on a GB300 with -m gpu)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_17018_gb300 import synth  # noqa: E402
from paper_2511_17018_gb300 import tpcfit as tf  # noqa: E402
from paper_2511_17018_gb300.frames import FrameBatch, GraphedFrameFit, fit_frames  # noqa: E402


def _bits(a, b):
    return all(np.array_equal(np.ascontiguousarray(a[k]).view(np.int32), np.ascontiguousarray(b[k]).view(np.int32))
               for k in ("params", "cov", "chi2", "ndf"))


def _host(out):
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.fixture(scope="module")
def frames():
    sizes = [1000, 3000, 257, 5000, 1800]
    return [synth.generate(n, 100 + i, drop_p=0.05, cap_lengths=True) for i, n in enumerate(sizes)]


def _individual(fitter, frames, aligns=None):
    outs = []
    for i, fr in enumerate(frames):
        if aligns is not None:
            fitter.set_alignment(aligns[i])
        outs.append(_host(fitter.fit(tf.frame_to_device(fr))))
    fitter.set_alignment(None)
    return {k: np.concatenate([o[k] for o in outs], axis=-1) for k in outs[0]}


@pytest.mark.parametrize("det", [True, False])
def test_frames_equal_individual_fits(frames, det):
    f = tf.Fitter(frames[0].geometry, frames[0].bz, deterministic=det)
    try:
        ref = _individual(f, frames)
        got = _host(fit_frames(f, FrameBatch.from_frames(frames)))
        assert _bits(got, ref)
        assert f.status()[0] == tf.OK
    finally:
        f.close()


def test_per_frame_alignment(frames):
    f = tf.Fitter(frames[0].geometry, frames[0].bz, deterministic=True)
    try:
        aligns = [torch.from_numpy(synth.alignment_offsets(200 + i)).cuda() for i in range(len(frames))]
        ref = _individual(f, frames, aligns)
        got = _host(fit_frames(f, FrameBatch.from_frames(frames), frame_alignment=torch.stack(aligns).contiguous()))
        assert _bits(got, ref)
    finally:
        f.close()


def test_graph_replay_and_in_place_refill(frames):
    f = tf.Fitter(frames[0].geometry, frames[0].bz, deterministic=True)
    try:
        batch = FrameBatch.from_frames(frames)
        g = GraphedFrameFit(f, batch)
        direct = _host(fit_frames(f, batch))
        assert _bits(_host(g.replay()), direct)
        # refill the seeds in place: the replay sees the new inputs
        batch.seeds[4].mul_(1.01)
        direct2 = _host(fit_frames(f, batch))
        assert _bits(_host(g.replay()), direct2)
        assert not _bits(direct, direct2)
    finally:
        f.close()


def test_ready_flags_streamed_frames(frames):
    # clusters arrive frame by frame from pinned host memory on a copy stream;
    # each frame's flag is set by a copy after its clusters: the persistent fit
    # waits per frame and ends with the same result as the resident batch
    f = tf.Fitter(frames[0].geometry, frames[0].bz, deterministic=True)
    try:
        full = FrameBatch.from_frames(frames)
        ref = _host(fit_frames(f, full))
        host = {k: getattr(full, k).cpu().pin_memory() for k in ("y", "z", "rowsec")}
        dev = {k: torch.zeros_like(getattr(full, k)) for k in ("y", "z", "rowsec")}
        batch = FrameBatch(dev["y"], dev["z"], dev["rowsec"], full.offsets, full.seeds, full.frame_base)
        nf = batch.n_frames
        flags = torch.zeros(nf, dtype=torch.int32, device="cuda")
        one = torch.ones(1, dtype=torch.int32).pin_memory()
        torch.cuda.synchronize()
        out = tf.empty_outputs(batch.n_tracks)
        fit_stream = torch.cuda.Stream()   # not the legacy default stream
        with torch.cuda.stream(fit_stream):
            fit_frames(f, batch, out, frame_ready=flags, wait_timeout_ns=2_000_000_000)
        copy = torch.cuda.Stream()
        off = full.offsets.cpu().numpy()
        fb = full.frame_base.cpu().numpy()
        with torch.cuda.stream(copy):
            for fi in range(nf):
                a, b = int(off[fb[fi]]), int(off[fb[fi + 1]])
                for k in ("y", "z", "rowsec"):
                    dev[k][a:b].copy_(host[k][a:b], non_blocking=True)
                flags[fi:fi + 1].copy_(one, non_blocking=True)
        torch.cuda.synchronize()
        st, code, trk = f.status(fit_stream)
        assert st == tf.OK, (st, code, trk)
        assert _bits(_host(out), ref)
        # flags with the legacy default stream are refused up front
        with pytest.raises(tf.TpcfitError) as e:
            fit_frames(f, batch, out, frame_ready=flags, stream=0)
        assert e.value.status == tf.EINVAL
    finally:
        f.close()


def test_ready_wait_runs_out_without_harm(frames):
    f = tf.Fitter(frames[0].geometry, frames[0].bz)
    try:
        batch = FrameBatch.from_frames(frames[:3])
        flags = torch.ones(3, dtype=torch.int32, device="cuda")
        flags[1] = 0                       # nothing ever sets this flag
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            out = fit_frames(f, batch, frame_ready=flags, wait_timeout_ns=50_000_000)
        out = _host(out)
        fb = batch.frame_base.cpu().numpy()
        st, code, trk = f.status(s)
        assert st == tf.ETIMEOUT and code == 3 and fb[1] <= trk < fb[2]
        assert np.all(out["ndf"][fb[1]:fb[2]] == -3)
        assert np.all(out["ndf"][: fb[1]] > 0) and np.all(out["ndf"][fb[2]:] > 0)
        # the context stays usable
        again = _host(fit_frames(f, batch))
        assert np.all(again["ndf"] > 0) and f.status()[0] == tf.OK
    finally:
        f.close()


def test_frames_from_pool_sampling():
    pool = synth.generate(3000, 7, drop_p=0.05, cap_lengths=True)
    rng = np.random.default_rng(8)
    picks = [rng.integers(0, pool.n_tracks, n) for n in (500, 1200, 40)]
    batch = FrameBatch.from_pool(pool, picks)
    f = tf.Fitter(pool.geometry, pool.bz, deterministic=True)
    try:
        got = _host(fit_frames(f, batch))
        whole = _host(f.fit(tf.frame_to_device(pool)))
        idx = np.concatenate(picks)
        for k in ("params", "chi2", "ndf"):
            a = got[k]
            b = whole[k][..., idx]
            assert np.array_equal(np.ascontiguousarray(a).view(np.int32), np.ascontiguousarray(b).view(np.int32)), k
    finally:
        f.close()


@pytest.mark.parametrize("lanes", [4, 16])
def test_frames_with_several_lanes_per_track(frames, lanes):
    # the batched launch with 32 / lanes tracks per warp: bit for bit the
    # one-lane per-frame fits (deterministic), and a ready wait that runs out
    # still marks exactly its frame
    f = tf.Fitter(frames[0].geometry, frames[0].bz, deterministic=True)
    try:
        ref = _individual(f, frames)
        f.set_config(lanes, 4, 24, True)
        batch = FrameBatch.from_frames(frames)
        assert _bits(_host(fit_frames(f, batch)), ref)
        flags = torch.ones(batch.n_frames, dtype=torch.int32, device="cuda")
        flags[2] = 0
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            out = fit_frames(f, batch, frame_ready=flags, wait_timeout_ns=20_000_000)
        out = _host(out)
        fb = batch.frame_base.cpu().numpy()
        assert f.status(s)[0] == tf.ETIMEOUT
        assert np.all(out["ndf"][fb[2]:fb[3]] == -3)
        keep = np.r_[0:fb[2], fb[3]:fb[-1]]
        assert np.array_equal(out["ndf"][keep], ref["ndf"][keep])
    finally:
        f.close()
