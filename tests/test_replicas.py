"""The N > 1 path of bench.py: independent replicas, one rank per GPU, no
data-path collective; the only exchange is the MAX all-reduce of the timed
region.  Run here as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [100.0, 150.0][rank]
    out[rank] = bench.job_throughput(64, ms, world)
    dist.destroy_process_group()


def test_job_throughput_two_gloo_ranks():
    world = 2
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        value, ms = out[r]
        assert ms == 150.0                      # the slowest rank's time
        assert abs(value - 2 * 64 / 0.150) < 1e-9  # all ranks' units over it


def test_job_throughput_single_rank():
    import bench
    value, ms = bench.job_throughput(64, 250.0, 1)
    assert ms == 250.0 and abs(value - 256.0) < 1e-12
