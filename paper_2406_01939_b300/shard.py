"""One trajectory's products sharded over ranks, and the collectives that join them.

Without node capacity the products of a fulfilment trajectory never interact
(Assumption 1 of Sec. 3.2): an order changes only its own product's stock row
and the policy sees only that row and the order's region.  So the orders of
disjoint product sets can be simulated on different GPUs, each by Picard
iteration over its own orders, and the pieces are the sequential path of the
whole trajectory.  Each rank owns the products `owner == rank`, balanced by
their demand (orders per product, largest first onto the least-loaded rank);
its sub-instance keeps those products' orders in time order with local product
ids.  After the simulation one all-reduce gives the trajectory's cost, lost
count and largest pass count, and an all-gather places every rank's actions at
their global times.  The Gumbel policy keys its noise by the order's time in
the whole trajectory, which a sub-instance does not carry: it is sharded by
trajectories instead (gradient_all_reduce).

Works with any torch.distributed backend: NCCL between GPUs, gloo on CPU.
"""
from __future__ import annotations

import numpy as np

from .synth import Instance


def product_shards(prod: np.ndarray, K: int, world: int) -> np.ndarray:
    """owner[k] of every product: products in decreasing order of their order
    count (ties by id) go to the rank with the fewest orders so far (lowest
    rank on ties).  Deterministic, so every rank computes the same table."""
    counts = np.bincount(np.asarray(prod, np.int64), minlength=K)
    order = np.lexsort((np.arange(K), -counts))
    load = np.zeros(world, np.int64)
    owner = np.empty(K, np.int32)
    for k in order:
        r = int(np.argmin(load))
        owner[k] = r
        load[r] += counts[k]
    return owner


def shard_instance(inst: Instance, owner: np.ndarray, rank: int):
    """The sub-instance of rank `rank`: its products' orders in time order with
    local product ids (the owned products in increasing id), their x0 and lam
    rows; regions and the cost table unchanged.  Returns (sub-instance, times of
    its orders in the trajectory, global ids of its products)."""
    if getattr(inst, "cap", None) is not None:
        raise ValueError("node capacity couples products: a trajectory with capacity is not sharded")
    mine = np.flatnonzero(owner == rank).astype(np.int32)
    local = np.full(inst.K, -1, np.int32)
    local[mine] = np.arange(mine.size, dtype=np.int32)
    times = np.flatnonzero(local[inst.prod] >= 0).astype(np.int64)
    K = max(1, int(mine.size))
    x0 = np.ascontiguousarray(inst.x0[mine] if mine.size else np.zeros((1, inst.N), np.int32))
    lam = None
    if inst.lam is not None:
        lam = np.ascontiguousarray(inst.lam[mine] if mine.size else np.zeros((1, inst.N), np.int32))
    sub = Instance(int(times.size), inst.N, K, inst.R,
                   np.ascontiguousarray(local[inst.prod[times]], dtype=np.int32),
                   np.ascontiguousarray(inst.reg[times], dtype=np.int32), x0,
                   np.ascontiguousarray(inst.cost), lam)
    return sub, times, mine


def join_scalars(total_cost: int, lost: int, iters: int, device=None):
    """All-reduce of one rank's (cost, lost) by sum and pass count by max: the
    trajectory's totals and the passes of its slowest shard."""
    import torch
    import torch.distributed as dist
    s = torch.tensor([int(total_cost), int(lost)], dtype=torch.int64, device=device)
    m = torch.tensor([int(iters)], dtype=torch.int64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return int(s[0]), int(s[1]), int(m[0])


def gather_actions(actions, times, T: int, device=None):
    """All-gather of every rank's actions (int8, in its orders' time order) into
    the trajectory's action array (int8 [T], every order written once)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size()
    a = torch.as_tensor(np.asarray(actions, np.int8)).to(device)
    t = torch.as_tensor(np.asarray(times, np.int64)).to(device)
    n = torch.tensor([a.numel()], dtype=torch.int64, device=device)
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n)
    width = int(max(int(x) for x in ns))
    pa = torch.full((width,), -2, dtype=torch.int8, device=device)
    pt = torch.full((width,), -1, dtype=torch.int64, device=device)
    pa[:a.numel()] = a
    pt[:t.numel()] = t
    ga = [torch.empty_like(pa) for _ in range(world)]
    gt = [torch.empty_like(pt) for _ in range(world)]
    dist.all_gather(ga, pa)
    dist.all_gather(gt, pt)
    out = torch.full((T,), -2, dtype=torch.int8, device=device)
    for r in range(world):
        k = int(ns[r])
        out[gt[r][:k]] = ga[r][:k]
    return out


def gradient_all_reduce(grad, objective: float, device=None):
    """Sum over ranks of the policy-gradient objective and its gradient (each
    rank holding its own trajectories' sums): the batch's J and dJ/dtheta."""
    import torch
    import torch.distributed as dist
    dist.all_reduce(grad, op=dist.ReduceOp.SUM)
    j = torch.tensor([float(objective)], dtype=torch.float64, device=device)
    dist.all_reduce(j, op=dist.ReduceOp.SUM)
    return grad, float(j[0])
