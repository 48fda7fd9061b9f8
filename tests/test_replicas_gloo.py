"""The multi-GPU form is replicas only: every rank registers its own image
pair and the job-level numbers are the max-over-ranks time and the summed
voxel throughput.  This checks that aggregation with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [100.0, 150.0][rank]
    n_local = [2 ** 24, 2 ** 24][rank]
    ms, value = bench.aggregate_ranks(ms_local, n_local, world, device="cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        ms, value = out[r]
        assert ms == 150.0  # the slowest rank sets the step time
        assert abs(value - 2 * 2 ** 24 / 0.150 / 1e9) < 1e-12  # all ranks' voxels


def test_single_rank_aggregation_is_local():
    import bench
    ms, value = bench.aggregate_ranks(80.0, 2 ** 24, 1)
    assert ms == 80.0 and abs(value - 2 ** 24 / 0.08 / 1e9) < 1e-12
