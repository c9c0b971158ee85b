"""Multi-rank host logic of the benchmark on CPU ranks (gloo, two
processes): the independent units (codes) are split among ranks exactly
once, and job times and counts combine as the slowest rank and the sum."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    bench.dist_init(world, 0, backend="gloo")
    mine = list(bench.shard(512, rank, world))
    slowest = bench.max_over_ranks(10.0 + rank, world)
    total = bench.sum_over_ranks(len(mine), world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out.put((rank, mine, slowest, total, gathered))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_shard_and_reduce_on_cpu_ranks(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mine, slowest, total, gathered in results:
        assert slowest == 10.0 + world - 1
        assert total == 512
        flat = [i for part in gathered for i in part]
        assert sorted(flat) == list(range(512))  # every code exactly once
        assert mine == gathered[rank] and mine == sorted(mine)


def test_shard_single_rank():
    import bench

    assert list(bench.shard(7, 0, 1)) == list(range(7))
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert [len(bench.shard(10, r, 4)) for r in range(4)] == [3, 3, 2, 2]
