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


# ------------------------------------------------ one volume split in z-slabs
def _slab_worker(rank, world, port, out):
    # each rank computes the outputs of its z-slab from its slab of the input
    # (grown by the halo, clipped to the volume); rank 0 gathers and stitches.
    # The per-rank compute here is the oracle (no GPU on this machine); on the
    # GPU the same slabs go through ct_run_box (bench.py --split zslab)
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_2508_07476_gb300 import partition, synth
    W = synth.single_chunk_64()
    vol, mask = synth.generate(W.spec)
    cen, ax = synth.frame_of(W.spec)
    nz, ny, nx = vol.shape
    h = O.radius(W.sigma) + O.radius(W.rho)
    sl = partition.z_slabs((nx, ny, nz), world, h)[rank]
    i0, i1 = sl.in_z
    z0, z1 = sl.out_z
    sub = np.ascontiguousarray(vol[i0:i1])
    msub = np.ascontiguousarray(mask[i0:i1])
    # positions of the slab's array are global ones shifted by i0 along z
    c_loc = (cen[0], cen[1], cen[2] - i0)
    part = O.pipeline(sub, W.sigma, W.rho, c_loc, ax, mask=msub, lo=(0, 0, z0 - i0), n=(nx, ny, z1 - z0))
    parts = [None] * world
    dist.all_gather_object(parts, (z0, z1, part))
    if rank == 0:
        out["parts"] = parts
        out["whole"] = O.pipeline(vol, W.sigma, W.rho, cen, ax, mask=mask)
    dist.barrier()
    dist.destroy_process_group()


def test_z_slabs_stitch_to_the_whole_volume():
    import numpy as np
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_slab_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    whole = out["whole"]
    covered = np.zeros(whole["fa"].shape[0], int)
    for z0, z1, part in out["parts"]:
        covered[z0:z1] += 1
        for k in ("S", "evals", "v", "fa"):  # independent of positions: bit for bit
            w = whole[k][..., z0:z1, :, :]
            np.testing.assert_array_equal(part[k], w, err_msg=k)
        for k in ("ha", "ia"):  # positions shifted by the slab origin: equal to FP64 rounding
            w = whole[k][z0:z1]
            np.testing.assert_allclose(part[k], w, rtol=0, atol=1e-9, equal_nan=True, err_msg=k)
    assert np.all(covered == 1)


def test_z_slab_partition_arithmetic():
    from paper_2508_07476_gb300 import partition
    for dims, world, h in [((8, 9, 64), 2, 16), ((5, 5, 7), 3, 40), ((4, 4, 100), 8, 12), ((3, 3, 2), 4, 5)]:
        slabs = partition.z_slabs(dims, world, h)
        assert len(slabs) == world
        nz = dims[2]
        z = 0
        for s in slabs:
            z0, z1 = s.out_z
            i0, i1 = s.in_z
            assert z0 == z and z1 >= z0
            z = z1
            assert s.out_n[:2] == dims[:2] and s.in_n[:2] == dims[:2]
            if z1 > z0:
                assert i0 == max(0, z0 - h) and i1 == min(nz, z1 + h)
        assert z == nz
        sizes = [s.out_n[2] for s in slabs]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        partition.z_slabs((4, 4, 4), 0, 1)
