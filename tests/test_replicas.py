"""Multi-GPU is replicas only: N independent factorizations, one per rank, with no collective on
the data path.  The ranks share host logic only: the barrier around the timed region, the
element-wise maximum of their wall times, and the whole-job rate (every rank's flops over the
slowest rank's time).  Two gloo ranks on the CPU check that logic as `bench.py` runs it."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        bench.barrier(world)
        walls = bench.gather_max(world, [1.0 + rank, 5.0 - 2.0 * rank])   # rank 1 is slower, then faster
        rate = bench.job_rate(world, 3.0e9, 2, walls[0])
        q.put((rank, walls, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_wall_and_the_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(r for r, _, _ in out) == [0, 1]
    for _, walls, rate in out:
        assert walls == [2.0, 5.0]                      # element-wise maximum over the ranks
        assert rate == pytest.approx(2 * 3.0e9 * 2 / 2.0 / 1e9)   # both ranks' flops over the slower wall


def test_one_rank_needs_no_process_group():
    import bench

    bench.barrier(1)
    assert bench.gather_max(1, [1.5, 2.5]) == [1.5, 2.5]
    assert bench.job_rate(1, 2.0e9, 4, 2.0) == pytest.approx(4.0)
