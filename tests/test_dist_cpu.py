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


def _replica_worker(rank, world, port, out):
    """One replica: rank r solves its own seeded instance with the FP64 oracle
    (the CPU stand-in for the device solve), then the bench's reductions
    combine the ranks' iteration counts and times."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import time
    import bench
    import oracle as O
    from paper_2605_29291_gb300 import workloads as W
    prob = O.Problem.from_data(W.random_qcqp(40, 3, seed=100 + rank))
    t0 = time.perf_counter()
    r = O.rapdb(prob, p=O.default_params("yx", tol=1e-6, max_iter=5000))
    dt = time.perf_counter() - t0
    t = bench.max_over_ranks(dt, world, torch.device("cpu"))
    it = bench.sum_over_ranks(float(r.iters), world, torch.device("cpu"))
    bench.barrier(world)
    out[rank] = (r.status, r.iters, float(prob.f(r.x)), dt, t, it)
    dist.destroy_process_group()


def test_two_replicas_on_gloo_match_single_process_solves():
    """Replicas only: two gloo ranks each solve their own instance with no
    data-path collective; every rank's result equals the same solve in a
    single process, and the whole-job throughput is the summed iterations
    over the slowest rank's time."""
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2605_29291_gb300 import workloads as W
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_replica_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        res = dict(out)
    iters = []
    for r in range(world):
        status, it_r, f_r, dt_r, t_max, it_sum = res[r]
        prob = O.Problem.from_data(W.random_qcqp(40, 3, seed=100 + r))
        ref = O.rapdb(prob, p=O.default_params("yx", tol=1e-6, max_iter=5000))
        assert status == ref.status == 0
        assert it_r == ref.iters and f_r == float(prob.f(ref.x))   # bit-identical replica
        iters.append(it_r)
        assert t_max >= dt_r
    assert res[0][4] == res[1][4] == max(res[0][3], res[1][3])
    assert res[0][5] == res[1][5] == float(sum(iters))
