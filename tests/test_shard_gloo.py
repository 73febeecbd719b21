"""One trajectory sharded by products over ranks, and the policy gradient sharded
by trajectories, with two and three gloo ranks on CPU.

Every rank builds the same seeded instance, keeps its products' orders
(paper_2406_01939_b300.shard), and runs Algorithm 1 on them; the CPU oracle's
Picard iteration stands in for the GPU call so that the partition and the
collectives are what is tested.  The joined result must be the sequential path
of the whole trajectory (products never interact without capacity, Assumption
1 of Sec. 3.2): every action at its time, the total cost and the lost count.
The gradient of the REINFORCE surrogate, each rank summing its own
trajectories, must all-reduce to the gradient of the whole batch."""
import os
import pickle
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2406_01939_b300 import shard, synth
from paper_2406_01939_b300.synth import Policy


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _instance(kind):
    inst = synth.make_instance(900, 8, 13, 7, seed=31, stock="poisson", fill=0.7, with_lam=True)
    mlp = synth.make_mlp(8, 7, seed=3) if kind == "mlp" else None
    return inst, Policy(kind, mlp=mlp)


def _rank_trajectory(rank, world, port, kind, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import oracle

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inst, pol = _instance(kind)
        owner = shard.product_shards(inst.prod, inst.K, world)
        sub, times, mine = shard.shard_instance(inst, owner, rank)
        res = oracle.picard_chunked(sub, pol, 16) if sub.T else None
        acts = res["actions"] if sub.T else np.zeros(0, np.int8)
        seq = oracle.seq_sim(sub, pol)
        cost, lost = (int(seq["total_cost"]), int(seq["lost"])) if sub.T else (0, 0)
        iters = res["iters"] if sub.T else 1
        tc, tl, ti = shard.join_scalars(cost, lost, iters)
        full = shard.gather_actions(acts, times, inst.T).numpy()
        out.put(pickle.dumps((rank, full, tc, tl, ti, acts, seq["actions"] if sub.T else acts,
                              seq["x_final"][:len(mine)] if sub.T else None, mine, owner)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run(target, world, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port) + args + (q,)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(pickle.loads(q.get(timeout=180)) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world,kind", [(2, "dual"), (3, "greedy"), (2, "mlp")])
def test_product_shards_join_to_the_sequential_path(world, kind):
    import oracle
    inst, pol = _instance(kind)
    want = oracle.seq_sim(inst, pol)
    res = _run(_rank_trajectory, world, kind)
    owner = res[0][9]
    assert np.bincount(owner, minlength=world).min() > 0  # every rank holds products
    loads = np.bincount(owner, weights=np.bincount(inst.prod, minlength=inst.K), minlength=world)
    assert loads.max() - loads.min() <= np.bincount(inst.prod).max()  # balanced by demand
    for rank, full, tc, tl, ti, acts, seq_acts, xf, mine, _ in res:
        np.testing.assert_array_equal(full, want["actions"])  # every rank holds the whole path
        assert tc == want["total_cost"] and tl == want["lost"]
        np.testing.assert_array_equal(acts, seq_acts)  # Picard's fixed point on the shard
        np.testing.assert_array_equal(xf, want["x_final"][mine])
        assert ti == max(r[4] for r in res)


def _rank_gradient(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import oracle
    from oracle import pg

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        B = 5
        mlp = synth.make_mlp(8, 6, seed=11)
        params = pg.bf16_params_f64(mlp)
        keys = list(params)
        local = {k: np.zeros_like(v) for k, v in params.items()}
        J = 0.0
        for b in range(rank, B, world):  # trajectories dealt round-robin
            inst = synth.make_instance(250 + 40 * b, 8, 6, 6, seed=50 + b, stock="poisson", fill=0.8)
            acts = oracle.seq_sim(inst, Policy("gumbel", mlp=mlp, seed=9, traj=b))["actions"]
            jb, gb = pg.surrogate(inst, params, acts)
            J += jb
            for k in keys:
                local[k] += gb[k]
        flat = torch.from_numpy(np.concatenate([local[k].ravel() for k in keys]))
        g, Jt = shard.gradient_all_reduce(flat, J)
        out.put(pickle.dumps((rank, g.numpy(), Jt)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_gradient_all_reduce_equals_the_whole_batch():
    import oracle
    from oracle import pg
    mlp = synth.make_mlp(8, 6, seed=11)
    params = pg.bf16_params_f64(mlp)
    keys = list(params)
    tot = {k: np.zeros_like(v) for k, v in params.items()}
    Jw = 0.0
    for b in range(5):
        inst = synth.make_instance(250 + 40 * b, 8, 6, 6, seed=50 + b, stock="poisson", fill=0.8)
        acts = oracle.seq_sim(inst, Policy("gumbel", mlp=mlp, seed=9, traj=b))["actions"]
        jb, gb = pg.surrogate(inst, params, acts)
        Jw += jb
        for k in keys:
            tot[k] += gb[k]
    want = np.concatenate([tot[k].ravel() for k in keys])
    res = _run(_rank_gradient, 2)
    for rank, g, Jt in res:
        np.testing.assert_allclose(g, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
        assert Jt == pytest.approx(Jw, rel=1e-12)


def test_shard_rejects_capacity_and_handles_empty_ranks():
    inst = synth.make_instance(50, 4, 2, 3, seed=1)
    owner = shard.product_shards(inst.prod, inst.K, 5)  # more ranks than products
    subs = [shard.shard_instance(inst, owner, r) for r in range(5)]
    assert sum(s[0].T for s in subs) == inst.T
    assert sorted(np.concatenate([s[1] for s in subs]).tolist()) == list(range(inst.T))
    assert any(s[0].T == 0 for s in subs)
    inst.cap = np.full(4, 10, np.int32)
    with pytest.raises(ValueError):
        shard.shard_instance(inst, owner, 0)
