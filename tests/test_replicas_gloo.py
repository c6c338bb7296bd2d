"""The multi-GPU benchmark runs independent replicas (a single solve does not shard):
each rank times its own solves and the job reports the total solves over the slowest
rank's time.  That combination is checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [100.0, 250.0][rank]
    e2e_local = [300.0, 200.0][rank]
    ms, e2e = bench.combine_over_ranks([ms_local, e2e_local])
    out[rank] = (ms, e2e, bench.total_throughput(steps=4, world=world, ms=ms))
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        ms, e2e, value = out[r]
        assert ms == 250.0 and e2e == 300.0
        assert value == pytest.approx(8 / 0.25)
