"""Host-side logic of the multi-rank benchmark path (one process per GPU,
independent right-hand sides, no data-path collective): two gloo ranks on
the CPU check the slowest-rank timing and the whole-job throughput."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank                      # rank 1 is the slow one
    t = bench.max_over_ranks(ms, world, torch.device("cpu"))
    v = bench.whole_job_value(world, 1000, 10.0, 2, t)
    out[rank] = (t, v)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, v = out[r]
        assert t == 150.0
        assert v == pytest.approx(world * 1000 * 10.0 * 2 / 0.150)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(12.5, 1, None) == 12.5
    assert bench.whole_job_value(1, 10, 3.0, 4, 1000.0) == pytest.approx(120.0)
