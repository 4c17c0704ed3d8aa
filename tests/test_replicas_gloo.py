"""Multi-process path of bench.py (replicas, one column per rank) on CPU with gloo.

The method is not sharded across GPUs: each rank advances its own column and
only the timing crosses ranks (max over ranks), so the job's throughput is
all ranks' site updates over the slowest rank's time.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, local = bench.dist_env()
    assert (w, r, local) == (world, rank, rank)
    my_ms = 10.0 + 5.0 * rank                 # rank 1 is the slower one
    ms = bench.max_over_ranks(my_ms, w)
    out[rank] = (ms, bench.aggregate_mlups(w, 1_000_000, 100, ms))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_timing_is_max_over_ranks(world):
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    expect_ms = 10.0 + 5.0 * (world - 1)
    for r in range(world):
        ms, value = out[r]
        assert ms == expect_ms
        assert value == pytest.approx(world * 1e6 * 100 / (expect_ms * 1e-3) / 1e6)
