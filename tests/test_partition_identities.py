"""The two identities the GPU partition walks rest on, checked on the CPU
against one pass of the oracle's Algorithm 1 (which replays every process from
s_1 literally), from random caches:

* any assignment without capacity: process m's stock of (k, n) before its
  order t is max(0, x0 - (C - O + F)), C the cached actions naming (k, n) before
  t, O those at m's own orders, F m's fresh ones, so each (product, process)
  pair is an independent chain;
* product partition with node capacity: node n has capacity before t in m's
  view iff the (c_n + own cached successes - own fresh actions)-th cached
  success at n comes at or after t, a cached action succeeding iff its rank
  among the cached actions of its (product, node) is below x0.

Both are restated here in plain Python, independently of the kernels."""
import bisect

import numpy as np
import pytest

import oracle
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.synth import Policy


def scores(inst, kind, k, r):
    s = inst.cost[r].astype(np.int64)
    if kind == "dual":
        s = s - inst.lam[k]
    return s


def argmin_feasible(s, feasible):
    best = -1
    for j in range(len(s)):
        if feasible[j] and (best < 0 or s[j] < s[best]):
            best = j
    return best


def chains_pass(inst, kind, proc, cache):
    """One pass for the assignment proc, no capacity, as (product, process) chains."""
    T, N = inst.T, inst.N
    lists = {}
    for t in range(T):
        if cache[t] >= 0:
            lists.setdefault((int(inst.prod[t]), int(cache[t])), []).append(t)
    new = np.empty(T, np.int8)
    units = {}
    for t in range(T):
        units.setdefault((int(inst.prod[t]), int(proc[t])), []).append(t)
    for (k, _m), orders in units.items():
        F = np.zeros(N, np.int64)
        O = np.zeros(N, np.int64)
        for t in orders:
            X = inst.x0[k].astype(np.int64) - F + O
            feas = [bisect.bisect_left(lists.get((k, j), []), t) < X[j] for j in range(N)]
            a = argmin_feasible(scores(inst, kind, k, int(inst.reg[t])), feas)
            new[t] = a
            if a >= 0:
                F[a] += 1
            if cache[t] >= 0:
                O[cache[t]] += 1
    return new


def products_capacity_pass(inst, kind, P, cache):
    """One pass of the product partition (k -> k mod P) with node capacity, from
    rank-based successes and the per-node lists of their times."""
    T, N = inst.T, inst.N
    seen = {}
    succ = np.zeros(T, bool)
    S = [[] for _ in range(N)]
    for t in range(T):
        c = int(cache[t])
        if c >= 0:
            key = (int(inst.prod[t]), c)
            rank = seen.get(key, 0)
            seen[key] = rank + 1
            if rank < inst.x0[key]:
                succ[t] = True
                S[c].append(t)
    new = np.empty(T, np.int8)
    for m in range(P):
        stock = {}
        delta = np.zeros(N, np.int64)
        for t in range(T):
            k = int(inst.prod[t])
            if k % P != m:
                continue
            xs = stock.setdefault(k, inst.x0[k].astype(np.int64).copy())
            feas = []
            for j in range(N):
                n = int(inst.cap[j]) + int(delta[j])
                cap_ok = n > 0 and (n > len(S[j]) or S[j][n - 1] >= t)
                feas.append(xs[j] > 0 and cap_ok)
            a = argmin_feasible(scores(inst, kind, k, int(inst.reg[t])), feas)
            new[t] = a
            if a >= 0:
                xs[a] -= 1
                delta[a] -= 1
            if succ[t]:
                delta[cache[t]] += 1
    return new


def random_cache(rng, T, N):
    return rng.integers(-1, N, T).astype(np.int8)


@pytest.mark.parametrize("seed", range(6))
def test_any_assignment_is_independent_chains(seed):
    rng = np.random.default_rng(seed)
    T, N, K = int(rng.integers(40, 160)), int(rng.integers(2, 7)), int(rng.integers(1, 6))
    inst = synth.make_instance(T, N, K, 4, seed=seed, stock="poisson", fill=0.5, with_lam=True)
    for kind in ("greedy", "dual"):
        for proc in (synth.uniform_assignment(T, int(rng.integers(1, 9)), seed=seed),
                     (np.arange(T) // max(1, T // 5)).astype(np.int32),
                     (inst.prod % 3).astype(np.int32)):
            for cache in (np.full(T, -1, np.int8), random_cache(rng, T, N)):
                want = oracle.picard_partition(inst, Policy(kind), proc, max_iters=1,
                                               alpha_init=cache)["actions"]
                np.testing.assert_array_equal(chains_pass(inst, kind, proc, cache), want)


@pytest.mark.parametrize("seed", range(6))
def test_product_partition_capacity_from_success_lists(seed):
    rng = np.random.default_rng(100 + seed)
    T, N, K = int(rng.integers(40, 160)), int(rng.integers(2, 7)), int(rng.integers(1, 7))
    inst = synth.make_instance(T, N, K, 4, seed=seed, stock="poisson", fill=0.7, with_lam=True)
    inst.cap = synth.node_capacity(T, N, seed=seed, frac=float(rng.uniform(0.2, 0.9)))
    for kind in ("greedy", "dual"):
        for P in (1, 2, K):
            for cache in (np.full(T, -1, np.int8), random_cache(rng, T, N)):
                want = oracle.picard_partition(inst, Policy(kind), (inst.prod % P).astype(np.int32),
                                               max_iters=1, alpha_init=cache)["actions"]
                np.testing.assert_array_equal(products_capacity_pass(inst, kind, P, cache), want)
