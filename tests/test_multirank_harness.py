"""The multi-rank benchmark harness on CPU ranks (gloo, world size 2): every
rank anneals its own instance (weak scaling, no data-path collective); the
reported value is all ranks' attempts over the slowest rank's time."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = [120.0, 250.0][rank]             # rank 1 is the slower one
    ms_max = bench.max_over_ranks(ms, dist, "cpu")
    dist.barrier()
    q.put((rank, ms_max, bench.aggregate_value(1e9, world, ms_max)))
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29511
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [250.0, 250.0]
    assert res[0][2] == pytest.approx(2 * 1e9 / 0.25)
