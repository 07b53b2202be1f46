"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.  Each rank
solves its own instance (weak scaling, no data-path collective); the bench
takes the maximum time and the summed iterations over ranks."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    # rank-dependent per-rank results: time 1.0 + rank, iterations 100 * (rank + 1)
    t = bench.max_over_ranks(1.0 + rank, world, torch.device("cpu"))
    it = bench.sum_over_ranks(100.0 * (rank + 1), world, torch.device("cpu"))
    bench.barrier(world)
    out[rank] = (t, it)
    dist.destroy_process_group()


def test_two_rank_aggregation_on_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        t, it = res[r]
        assert t == 2.0              # max over ranks
        assert it == 300.0           # 100 + 200
    # whole-job throughput as bench.py reports it: summed iterations / slowest rank
    assert res[0][1] / res[0][0] == 150.0


def test_single_rank_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.sum_over_ranks(7.0, 1, None) == 7.0
