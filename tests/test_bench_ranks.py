"""bench.py's multi-rank path on the CPU: two gloo ranks, each timing its own
replica purifications; rank aggregation takes the maximum and the whole-job
value divides by all purifications of all ranks."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [100.0 + 10 * rank, 110.0 + 10 * rank, 120.0 + 30 * rank]
    got = bench.max_over_ranks(local, dist, "cpu")
    value, e2e = bench.per_purification(got[:2], world, steps=2)
    out.put((rank, got, value, e2e))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value, e2e in res:
        assert got == [110.0, 120.0, 150.0]
        assert value == pytest.approx(110.0 / 4)
        assert e2e == pytest.approx(120.0 / 4)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.0, 2.0]) == [1.0, 2.0]
    assert bench.per_purification([10.0], 1, 5) == [2.0]
