"""Replica aggregation of bench.py across ranks (gloo, world size 2, CPU).

With N GPUs bench.py runs one independent replica per rank; rank 0 reports
the total states of all ranks over the slowest rank's time.  These are the
host-side collectives it uses.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    bench.dist_init(world, use_cuda=False)
    states = 1000.0 * (rank + 1)
    ms = 10.0 + 5.0 * rank
    bench.barrier()
    out[rank] = (bench.reduce_scalar(states, "sum"), bench.reduce_scalar(ms, "max"))
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    port = _free_port()
    with tmp.Manager() as mgr:
        out = mgr.dict()
        tmp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        got = dict(out)
    assert got[0] == got[1] == (3000.0, 15.0)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_scalar(7.0, "max") == 7.0
    assert bench.reduce_scalar(7.0, "sum") == 7.0
    assert bench.dist_env() == (0, 1, 0) or "RANK" in os.environ
