"""The N > 1 host path of bench.py on CPU: two gloo ranks, each with its own
timing, agree on the slowest rank's time and on the whole-job rate (weak
scaling: units of all ranks over the max time)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        assert bench.dist_env() == (world, rank, rank)
        seconds = 0.5 + rank  # rank 1 is the slow one
        q.put((rank, bench.max_over_ranks(seconds), bench.job_rate(1000, seconds, world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, mx, rate in got:
        assert mx == 1.5
        assert rate == pytest.approx(1000 * world / 1.5)


def test_single_process_is_its_own_max():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(0.25) == 0.25
    assert bench.job_rate(100, 0.5, 1) == 200
