"""The multi-rank bench path on CPU: two gloo ranks (world size 2) run the
bench's whole-job aggregation - the job time is the slowest rank's and the
units are summed over the replicas - and only rank 0 would print."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs, units = bench.job_totals(1.0 + rank, 480.0 * (rank + 1), world, "cpu")
    out[rank] = (secs, units)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        assert out[0] == (2.0, 1440.0) and out[1] == (2.0, 1440.0)


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(1.5, 480.0, 1) == (1.5, 480.0)
