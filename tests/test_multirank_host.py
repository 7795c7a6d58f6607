"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The operator runs as independent replicas, one per GPU (weak scaling, no
collective on the data path); the only cross-rank step is the timing: the
job's step time is the slowest rank's, and the whole-job throughput is
world x 1000 / that time.
"""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]
    got = bench.max_over_ranks(ms, "cpu", world)
    out[rank] = (got, bench.job_throughput(got, world))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (20.0, 100.0)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(7.5, "cpu", 1) == 7.5
    assert bench.job_throughput(20.0, 1) == pytest.approx(50.0)
