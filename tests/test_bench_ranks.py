"""The multi-rank timing logic of bench.py (max over ranks, whole-job rate) on two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    mx = bench.max_over_ranks(10.0 + 5.0 * rank, world, device="cpu")
    rate = bench.whole_job_rate(64, world, mx)
    out.put((rank, mx, rate))
    dist.destroy_process_group()


def test_timing_is_the_slowest_rank_and_value_counts_every_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [15.0, 15.0]
    assert all(abs(g[2] - 2 * 64 / 15.0) < 1e-12 for g in got)


def test_single_rank_passes_through():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(32, 1, 2.0) == 16.0
