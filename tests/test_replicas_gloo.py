"""The multi-rank bench path on CPU: two gloo ranks, each timing its own replica.

bench.py runs one replica per GPU (the single-graph path does not shard); the job's time is the
slowest rank's and its work the sum over ranks. This checks that aggregation with world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as mp


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
    import bench
    ms = [120.0, 95.0][rank]          # per-rank timed milliseconds
    edges = [1e9, 2e9][rank]           # per-rank LP edges
    out[rank] = (bench.max_over_ranks(ms, dist), bench.sum_over_ranks(edges, dist))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (120.0, 3e9)
