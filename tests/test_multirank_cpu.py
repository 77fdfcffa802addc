"""The N-GPU bench path is N independent replicas (rays are independent and
objects read-only, so nothing is exchanged): each rank renders its own full
workload and only the timing is combined -- a barrier and the maximum over
ranks.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = [0.25, 0.75][rank]            # per-rank timed seconds
    bench._barrier(world)
    tmax = bench._max_over_ranks(t, world, device="cpu")
    out[rank] = (tmax, bench.replica_throughput(1000.0, tmax, world))
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_timing():
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
        tmax, thr = out[r]
        assert tmax == 0.75                 # every rank sees the slowest rank's time
        assert thr == pytest.approx(2000.0 / 0.75)  # weak scaling: all ranks' units / max time


def test_single_rank_is_identity():
    import bench
    assert bench._max_over_ranks(1.5, 1) == 1.5
    assert bench.replica_throughput(10.0, 2.0, 1) == 5.0
