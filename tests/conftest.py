import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); run with -m gpu")


@pytest.fixture(scope="session")
def synth():
    from paper_2511_17018_gb300 import synth as s
    return s


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    return oracle


@pytest.fixture(scope="session")
def frame_small(synth):
    """1,000 tracks, natural lengths (the plain-fit workload)."""
    return synth.plain_frame()


@pytest.fixture(scope="session")
def frame_drop(synth):
    """4,000 tracks with 5% drop and the U{10..152} length cap."""
    return synth.generate(4000, 2, drop_p=0.05, cap_lengths=True)


def truth_trajectory(oracle, frame):
    """Exact state at every hit: the first-hit truth carried hit to hit by the
    FP64 propagator (used as the linearisation reference)."""
    g = frame.geometry
    off = frame.offsets.astype(np.int64)
    rs = frame.rowsec.astype(np.int64)
    ref = np.zeros((frame.n_hits, 5))
    for i in range(frame.n_tracks):
        a, b = off[i], off[i + 1]
        p = frame.truth[:, i].copy()
        ref[a] = p
        x = g.row_x[rs[a] >> 6]
        sec = rs[a] & 63
        for j in range(a + 1, b):
            p, x, _ = oracle.step(g, frame.bz, p, x, sec, rs[j] >> 6, rs[j] & 63)
            sec = rs[j] & 63
            ref[j] = p
    return ref
