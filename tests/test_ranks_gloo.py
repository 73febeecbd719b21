"""The multi-rank reduction of bench.py on CPU: two gloo ranks (world size 2).

Each rank simulates its own synthetic workload (weak scaling, no collective on
the data path); the job's rate is the units of all ranks over the slowest
rank's timed total.  Here every rank runs the oracle's sequential simulation of
a small seeded instance (CPU) and reports a made-up timed total, so the
reduction can be checked exactly."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import oracle
    from paper_2406_01939_b300 import synth

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = bench.rank_seed(7, rank)
        T = 300 + 100 * rank  # ranks need not hold the same number of orders
        inst = synth.make_instance(T, 8, 5, 6, seed=seed, stock="poisson", fill=0.9, with_lam=True)
        want = oracle.seq_sim(inst, synth.Policy("dual"))
        t_ms = 10.0 + 5.0 * rank  # rank 1 is the slowest
        rate, t_job = bench.job_rate(T, 3, t_ms, world)
        tot_cost = bench.over_ranks(want["total_cost"], world, "sum")
        out.put((rank, seed, T, rate, t_job, tot_cost, int(want["total_cost"]),
                 want["actions"][:50].tobytes()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_reduction():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = [r[1] for r in res]
    assert seeds == [7, 8]  # one workload per rank
    assert res[0][7] != res[1][7]  # different instances, different paths
    units = sum(r[2] for r in res) * 3
    for r in res:
        assert r[4] == 15.0  # max over ranks
        assert r[3] == pytest.approx(units / 0.015)  # every rank holds the job's rate
        assert r[5] == sum(x[6] for x in res)


def test_single_rank_is_identity():
    rate, t = bench.job_rate(1000, 4, 20.0, 1)
    assert t == 20.0 and rate == pytest.approx(4000 / 0.02)
    assert bench.over_ranks(3.5, 1, "sum") == 3.5
