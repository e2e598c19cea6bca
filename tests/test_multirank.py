"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

Each rank processes its own volume (weak scaling, no collective on the data
path); the only collective is the reduction of the step time to its maximum.
"""
import os
import socket

import pytest
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
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    m = bench.max_over_ranks(ms, world, device="cpu")
    out[rank] = (m, bench.job_voxels_per_s(512 ** 3, world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_max_time_and_job_throughput():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert out[0] == out[1]
    m, v = out[0]
    assert m == 15.0
    assert v == pytest.approx(2 * 512 ** 3 / 15e-3)
