"""Multi-rank path of bench.py on CPU: two gloo ranks run independent replicas and the
whole-job figures are the max-over-ranks time and the sum of points (the N > 1 launch
under torchrun uses the same collectives over NCCL)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.env_rank()[:2] == (rank, world)
        q.put((rank, bench.reduce_over_ranks(1.5 + rank, 1000 * (rank + 1), world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_sum_points():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(world))
    for r in range(world):
        assert got[r] == (2.5, 3000.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(3.0, 7, 1) == (3.0, 7.0)

