"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

Every rank advances independent runs; the only collectives are a barrier and
the maximum of the elapsed times.  The sharding of an ensemble must cover
every run exactly once.
"""
import os

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    t = bench.max_over_ranks(world, 1.5 + rank)
    mine = list(bench.shard(513, world, rank))
    q.put((rank, t, mine))
    dist.destroy_process_group()


def test_two_ranks_time_is_max_and_shards_cover_runs():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert all(t == 2.5 for _, t, _ in res)
    runs = res[0][2] + res[1][2]
    assert sorted(runs) == list(range(513))
    assert abs(len(res[0][2]) - len(res[1][2])) <= 1


@pytest.mark.parametrize("n,world", [(512, 1), (512, 8), (7, 3), (1, 4)])
def test_shard_partition(n, world):
    import bench
    allr = [i for r in range(world) for i in bench.shard(n, world, r)]
    assert sorted(allr) == list(range(n))
