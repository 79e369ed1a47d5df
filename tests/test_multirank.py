"""Host logic of the multi-GPU bench path (one replica per rank, no data
exchange): the job time is the slowest rank's, the value counts every
rank's cells.  Two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = bench.reduce_max_ms(times[rank], world, "cpu")
    out[rank] = (ms, bench.job_value(1000, 10, world, ms))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_timing_takes_the_slowest_rank(world):
    times = [12.5, 31.25][:world]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r][0] == max(times)
        assert res[r][1] == world * 1000 * 10 / (max(times) * 1e-3)


def test_single_rank_is_unchanged():
    import bench
    assert bench.reduce_max_ms(7.0, 1, "cpu") == 7.0
    assert bench.job_value(64, 3, 1, 2.0) == 64 * 3 / 2e-3
