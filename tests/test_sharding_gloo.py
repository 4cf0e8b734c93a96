"""Multi-rank host logic of the env-sharded benchmark, on CPU with gloo."""
import os

import pytest

from paper_2503_18616_gb300 import sharding


def test_env_ranges_partition_the_envs():
    for n, world in [(4096, 2), (1024, 3), (7, 4), (5, 8)]:
        ranges = [sharding.env_range(n, world, r) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        for (a, b), (c, d) in zip(ranges, ranges[1:]):
            assert b == c
        sizes = [b - a for a, b in ranges]
        assert max(sizes) - min(sizes) <= 1


def test_rank_seeds_are_distinct():
    assert len({sharding.rank_seed(7, r) for r in range(8)}) == 8


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = 1.0 + rank                      # rank 1 is the slowest
    tmax = sharding.max_over_ranks(t, dist, "cpu")
    out.put((rank, tmax, sharding.throughput(4096, world, 100, tmax), sharding.rank_seed(0, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_max_time_and_throughput():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]             # max over ranks
    assert res[0][2] == pytest.approx(2 * 4096 * 100 / 2.0)
    assert res[0][3] != res[1][3]
