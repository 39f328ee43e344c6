"""The seeded input generator follows the stated workload recipe (CPU).

The generator holds none of the fit's arithmetic; these tests check that its
frames have the distributions and structure the benchmark workloads are
defined by: pt log-uniform on [0.2, 10] GeV/c, |eta| < 0.9, charges +-1 with
equal odds, z0 ~ N(0, 5 cm), 5% of the clusters dropped, lengths capped at
U{10..152}, one cluster per crossed row in row order, sector and side
consistent with the track."""
import math

import numpy as np
import pytest

from paper_2511_17018_gb300 import synth

stats = pytest.importorskip("scipy.stats")


@pytest.fixture(scope="module")
def frame():
    return synth.generate(20000, 2, drop_p=0.05, cap_lengths=True)


def test_track_parameter_distributions(frame):
    qpt, tanl = frame.truth[4], frame.truth[3]
    pt = 1.0 / np.abs(qpt)
    u = (np.log(pt) - math.log(0.2)) / (math.log(10.0) - math.log(0.2))
    assert u.min() >= 0.0 and u.max() <= 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    eta = np.arcsinh(tanl)
    assert np.abs(eta).max() < 0.9
    assert stats.kstest((eta + 0.9) / 1.8, "uniform").pvalue > 1e-3
    assert abs(np.mean(qpt > 0) - 0.5) < 0.02


def test_lengths_drops_and_row_order(frame):
    lens = frame.lengths()
    assert lens.min() >= 10 and lens.max() <= 152
    rs = frame.rowsec.astype(np.int64)
    row, sec = rs >> 6, rs & 63
    assert sec.max() < 36 and row.max() < 152
    off = frame.offsets.astype(np.int64)
    first = np.zeros(frame.n_hits, bool)
    first[off[:-1]] = True
    assert np.all(np.diff(row)[~first[1:]] > 0)  # rows strictly ascending within a track
    # natural lengths: almost every track reaches row 115 or beyond (|eta| < 0.9, pt >= 0.2)
    nat = synth.generate(4000, 12, drop_p=0.05)
    r = (nat.rowsec.astype(np.int64) >> 6)
    o = nat.offsets.astype(np.int64)
    span = r[o[1:] - 1] - r[o[:-1]] + 1
    kept = np.diff(o)
    assert np.mean(r[o[1:] - 1] >= 115) > 0.97
    # 5% of the crossed rows are dropped
    assert abs(1.0 - kept.sum() / span.sum() - 0.05) < 0.005
    # caps U{10..152}: the capped frame's lengths spread over the whole range
    assert np.mean(lens < 40) > 0.1 and np.mean(lens > 120) > 0.05


def test_vertex_side_and_sector_geometry():
    fr = synth.generate(3000, 13, smear=0.0)
    rs = fr.rowsec.astype(np.int64)
    row, sec = rs >> 6, rs & 63
    # side: sectors 18-35 hold the clusters with z < 0
    assert np.all((sec >= 18) == (fr.z64 < 0.0))
    # every cluster lies inside its sector's coverage of its row
    xr = fr.geometry.row_x[row]
    assert np.all(np.abs(fr.y64) <= xr * math.tan(math.radians(10.0)) + 1e-9)
    assert np.all(np.abs(fr.z64) <= 250.0)
    # the vertex and azimuth draws
    rng = np.random.default_rng(5)
    q, tanl, phi0, zv = synth.draw_track_params(rng, 200000)
    assert abs(zv.std() - 5.0) < 0.05 and abs(zv.mean()) < 0.05
    assert stats.kstest(phi0 / (2 * math.pi), "uniform").pvalue > 1e-3


def test_frame_batch_gathers_pool_tracks_on_the_host():
    torch = pytest.importorskip("torch")
    from paper_2511_17018_gb300.frames import FrameBatch
    pool = synth.generate(800, 4, drop_p=0.05, cap_lengths=True)
    sizes = synth.frame_sizes_batched(4, 6, 20, 400)
    rng = np.random.default_rng(9)
    picks = [rng.integers(0, pool.n_tracks, int(s)) for s in sizes]
    b = FrameBatch.from_pool(pool, picks, device="cpu")
    owner = np.concatenate(picks)
    ref = pool.subset(owner)
    assert b.n_frames == 6 and b.n_tracks == owner.size
    assert np.array_equal(b.frame_base.numpy(), np.concatenate([[0], np.cumsum(sizes)]))
    assert np.array_equal(b.offsets.numpy(), ref.offsets)
    assert np.array_equal(b.y.numpy(), ref.y) and np.array_equal(b.z.numpy(), ref.z)
    assert np.array_equal(b.rowsec.numpy().view(np.uint16), ref.rowsec)
    assert np.array_equal(b.seeds.numpy(), ref.seeds)
    assert isinstance(b.y, torch.Tensor)
