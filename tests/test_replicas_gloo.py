"""The N > 1 path of bench.py (independent replicas, weak scaling): max-over-ranks timing and
whole-job throughput, exercised with two gloo ranks on CPU."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [2.0, 3.0][rank]          # the slower rank decides
    units = 1000.0                      # cell-steps processed by each rank
    t, value = bench.aggregate(elapsed, units, world, device="cpu")
    dist.barrier()
    q.put((rank, t, value))
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert all(p.exitcode == 0 for p in procs)
    for rank, t, value in out:
        assert t == 3.0
        assert value == pytest.approx(2 * 1000.0 / 3.0)
