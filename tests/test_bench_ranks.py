"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the whole-job
time is the slowest rank's, throughputs are world size x the slowest rank, and
ranks draw different batches."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    step_ms = [4.0, 6.5][rank]
    rates = [[100.0, 10.0], [80.0, 12.0]][rank]
    t, r = bench.combine_ranks(dist, torch, "cpu", step_ms, rates)
    q.put((rank, t, r, bench.rank_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, t, r, seed in res:
        assert t == 6.5                        # slowest rank
        assert r == [160.0, 20.0]              # world x slowest per-rank rate
    assert res[0][3] != res[1][3]              # different batches per rank
