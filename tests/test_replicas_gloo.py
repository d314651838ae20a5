"""The N > 1 path of the benchmark on CPU: replicas only (independent
right-hand sides, no data-path collective), so the only cross-rank steps are
the max of the step time over ranks and the whole-job rate.  Two gloo ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, dist, "cpu")    # rank 1 is the slow replica
    out[rank] = (ms, bench.whole_job_rate(168, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, rate = res[r]
        assert ms == 150.0
        assert rate == pytest.approx(168 * 2 / 0.150, rel=1e-15)


def test_single_process_without_group():
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.whole_job_rate(168, 1, 1000.0) == 168.0
