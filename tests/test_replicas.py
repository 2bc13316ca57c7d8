"""The multi-GPU layout (independent replicas) with two gloo ranks on the
CPU: distinct point sets per rank, the step time is the slowest rank's on
every rank, and the job throughput counts all ranks' points."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads as W
from paper_0904_3151_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = W.WORKLOADS["small"]
    X = W.clustered(500, wl.dim, 5, wl.sigma, replicas.replica_seed(wl.data_seed, rank))
    ms = replicas.max_over_ranks(10.0 + 3.0 * rank, dist)
    out[rank] = (float(X[0, 0]), ms, replicas.job_throughput(world, 500, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_own_distinct_sets():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0][0] != res[1][0]                       # different point sets
    assert res[0][1] == res[1][1] == 13.0               # the slowest rank's time
    assert res[0][2] == pytest.approx(2 * 500 / 0.013)


def test_single_process_is_identity():
    assert replicas.max_over_ranks(4.5) == 4.5
    assert replicas.replica_seed(1002, 0) == 1002
    assert replicas.job_throughput(1, 1000, 500.0) == 2000.0
