"""The multi-GPU benchmark runs one independent replica per rank and reduces only its
timing: the whole-job time is the slowest rank's and the work is the sum over ranks.
Checked with two gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bench.replica_totals(10.0 + 5.0 * rank, 1000 * (rank + 1), dist, torch.device("cpu"))
    out[rank] = (ms, units)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_totals_two_gloo_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in range(2):
        assert out[r] == (15.0, 3000.0)


def test_replica_totals_single_rank():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.replica_totals(7.0, 123, None, None) == (7.0, 123)
