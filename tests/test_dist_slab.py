"""x-slab decomposition with halo exchange (paper_0807_0602_gb300.slab) on CPU
ranks: two gloo processes, each stepping its slab, exchanging edge columns
by point-to-point send/recv after every step, reproduce the undivided run
bit for bit.

No GPU is needed: the slabs' lattices here are a test double over the FP64
oracle (the decomposition, the column bookkeeping and the exchange are the
product's host code; tests/test_gpu_slab.py runs the same decomposition on
the GPU library).
"""
import os

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 12


class OracleColumns:
    """Test double of the lattice interface the slabs use (step, get_columns,
    set_columns) over the FP64 oracle."""

    def __init__(self, run):
        import oracle
        self.o = oracle.OracleLattice(run["geom"], run["params"], run["init"][1], run["init"][2])

    def step(self, n=1):
        self.o.step(n)

    def get_columns(self, x0, n):
        return torch.from_numpy(np.ascontiguousarray(self.o.populations()[..., x0:x0 + n]))

    def set_columns(self, x0, buf):
        F = self.o.populations()
        F[..., x0:x0 + buf.shape[-1]] = buf.numpy()
        self.o.set_populations(F)

    def populations(self):
        return self.o.populations()


def _case():
    import workloads as W
    geom = W.capillary_geometry(40, 11, 8, 33, 0, 10)
    nA, nB = W.random_fields(geom, 5, 0.2, 1.2)
    return dict(geom=geom, params=W.params(1.1, 1.0, 0.8, -0.2, 0.1), init=("fields", nA, nB)), nA, nB


def _reference(run, steps):
    import oracle
    o = oracle.OracleLattice(run["geom"], run["params"], run["init"][1], run["init"][2])
    o.step(steps)
    return o.populations()


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_0807_0602_gb300 import slab as SL
    run, nA, nB = _case()
    sr = SL.SlabRank(run, nA, nB, factory=OracleColumns)
    sr.step(STEPS)
    q.put((rank, sr.slab.x0, sr.slab.x1, sr.slab.owned(sr.slab.lat.populations())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_undivided_run_bit_for_bit():
    import sys
    sys.path.insert(0, ROOT)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in range(2)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    run, _, _ = _case()
    want = _reference(run, STEPS)
    assert res[0][1] == 0 and res[0][2] == res[1][1] and res[1][2] == run["geom"]["nx"]
    got = np.concatenate([r[3] for r in res], axis=-1)
    assert np.array_equal(got, want)


def _leaving_worker(rank, world, port, q):
    """Rank 1 leaves between steps (after 3 steps and their exchanges, with
    nothing in flight); rank 0 steps on and must see its next exchange fail
    instead of waiting forever."""
    import sys
    import time
    from datetime import timedelta
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=10))
    from paper_0807_0602_gb300 import slab as SL
    run, nA, nB = _case()
    sr = SL.SlabRank(run, nA, nB, factory=OracleColumns)
    sr.step(3)
    if rank == 1:
        q.put((rank, "left", 0.0))
        q.close()
        q.join_thread()                  # the message is sent before the process vanishes
        os._exit(0)                      # no destroy_process_group: the peer just disappears
    t0 = time.monotonic()
    try:
        sr.step(3)
        q.put((rank, "no error", time.monotonic() - t0))
    except RuntimeError as e:            # gloo reports the lost peer (closed connection or timeout)
        q.put((rank, "error: " + str(e).splitlines()[0][:80], time.monotonic() - t0))
    q.close()
    q.join_thread()
    os._exit(0)


def test_a_rank_that_leaves_makes_the_next_exchange_fail_not_hang():
    import sys
    sys.path.insert(0, ROOT)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 28700 + os.getpid() % 1000
    procs = [ctx.Process(target=_leaving_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r[0], r[1:]) for r in (q.get(timeout=120) for _ in range(2)))
    for p in procs:
        p.join(timeout=60)
    assert res[1][0] == "left"
    assert res[0][0].startswith("error"), res[0]
    assert res[0][1] < 60.0


@pytest.mark.parametrize("parts", [1, 3, 4])
def test_slabs_of_one_process_reproduce_the_undivided_run(parts):
    from paper_0807_0602_gb300 import slab as SL
    run, nA, nB = _case()
    bounds = SL.slab_bounds(run["geom"]["nx"], parts)
    slabs = [SL.Slab(run, a, b, nA, nB, factory=OracleColumns) for a, b in bounds]
    SL.step_local(slabs, STEPS)
    got = np.concatenate([s.owned(s.lat.populations()) for s in slabs], axis=-1)
    assert np.array_equal(got, _reference(run, STEPS))


def test_a_slab_that_skips_the_exchange_differs():
    """The exchange matters: without it the halos go stale and the edge
    columns drift from the undivided run after a few steps."""
    from paper_0807_0602_gb300 import slab as SL
    run, nA, nB = _case()
    slabs = [SL.Slab(run, a, b, nA, nB, factory=OracleColumns) for a, b in SL.slab_bounds(run["geom"]["nx"], 2)]
    for _ in range(STEPS):
        for s in slabs:
            s.step()
    got = np.concatenate([s.owned(s.lat.populations()) for s in slabs], axis=-1)
    assert not np.array_equal(got, _reference(run, STEPS))


def test_slab_bounds_cover_the_grid():
    from paper_0807_0602_gb300 import slab as SL
    for nx, parts in ((40, 2), (41, 3), (8192, 8), (16, 4)):
        b = SL.slab_bounds(nx, parts)
        assert b[0][0] == 0 and b[-1][1] == nx and all(b[i][1] == b[i + 1][0] for i in range(parts - 1))
        assert max(x1 - x0 for x0, x1 in b) - min(x1 - x0 for x0, x1 in b) <= 1
    with pytest.raises(ValueError):
        SL.slab_bounds(7, 2)
