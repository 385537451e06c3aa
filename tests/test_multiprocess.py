"""The multi-rank host logic of bench.py on CPU with gloo (world size 2):
independent replicas get distinct seeds, and the job throughput takes the
slowest rank's step time and the sum of all ranks' units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [2.0, 3.0][rank]
    units = [100.0, 140.0][rank]
    value, ms = bench.job_throughput(ms_local, units, dist)
    out[rank] = (value, ms, bench.replica_seeds("knn_gmm", rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_job_throughput_and_replica_seeds():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, ms, seeds = res[rank]
        assert ms == 3.0
        assert abs(value - 240.0 / 3e-3) < 1e-6
    assert res[0][2] != res[1][2]
    assert res[0][2][0] == 1001  # rank 0 runs the named workload's own seed


def test_single_process_throughput():
    import bench
    value, ms = bench.job_throughput(4.0, 200.0, None)
    assert ms == 4.0 and value == 200.0 / 4e-3
