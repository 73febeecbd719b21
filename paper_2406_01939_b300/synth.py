"""Seeded synthetic fulfillment-optimization (FO) workloads.

Input generation only: this module draws order streams, inventories, cost
tables, dual prices and MLP parameters from a seeded numpy ``Generator(PCG64)``.
It holds none of the simulation or policy arithmetic, so both the CUDA path and
the CPU oracle may consume what it produces.

The paper's own instances (Appendix A.3: 30 population-weighted nodes, zip-code
distance rewards) rest on data that is not available; these generators stand in
for them with the shapes of the paper's FO experiments (Sec. 4): many products
with heavy-tailed demand Q_i proportional to i^beta (Sec. 4.1, Table 1), a few
dozen nodes, per-(region, node) fulfilment costs.

Named workloads (sizes as the benchmark and tests use them):
  greedy_small    T=4,096 orders, N=8 warehouses, K=16 products, R=32 regions,
                  x0 ~ U{0..20}, cost ~ U{1..100}, greedy policy, 64 chunks.
  dual_large      T=2^20, N=64, K=10,000, R=1,000, x0 ~ Poisson(1.05 T p_k / N),
                  lambda ~ U{0..30}, cost ~ U{1..100}, bid-price policy.
  mlp_medium      T=2^18, N=64, K=2,000, R=500, same inventory recipe, MLP policy
                  Linear(2N+16, 256)-ReLU-Linear(256, N), BF16 N(0, 0.02) params.
  batch_uneven    512 trajectories, T_i ~ U{16,384..262,144}, N=32, K=2,000,
                  R=200; even index greedy, odd index MLP.
  pg_large        64 trajectories of T=2^20, N=64, K=10,000, R=1,000, Gumbel MLP.
  capacity_large  dual_large plus node capacity c_1 for 80% of the orders, spread
                  pro rata to log-normal(0, 0.5) node weights (Sec. 3 model).
Product demand is a finite Zipf(1.1): p_k proportional to (k+1)^-1.1, product 0
the most popular; regions are uniform.

OWMR inventory control (Appendix B): one central warehouse, N retailers.
  owmr_base       one year of one product selling about 10,000 units a day over
                  4,000 stores (Appendix B.3): T = 3,650,000 unit demands, store
                  n drawn with weight (1 - a)^n (a = 0: uniform), stores reorder
                  at 10 units up to 20 (capacity 24), central (s, S) =
                  (1,000, 71,000), about one central replenishment a week;
                  two-hidden-layer network of width 512, BF16 N(0, 0.02), fed
                  (post-demand stock, demand, steps since the store's
                  previous demand / 4096).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

EMB = 16  # width of the region embedding fed to the MLP policy
HIDDEN = 256


@dataclass
class Instance:
    """One FO trajectory's inputs (all host numpy arrays, C-contiguous)."""

    T: int
    N: int
    K: int
    R: int
    prod: np.ndarray  # int32 [T]   product of order t
    reg: np.ndarray  # int32 [T]   region of order t
    x0: np.ndarray  # int32 [K, N] initial inventory
    cost: np.ndarray  # int32 [R, N] fulfilment cost
    lam: Optional[np.ndarray] = None  # int32 [K, N] dual prices (bid-price policy)
    cap: Optional[np.ndarray] = None  # int32 [N] node capacity c_1 (None: no capacity)


@dataclass
class MLPParams:
    """BF16 parameters stored as uint16 bit patterns.

    W1 [2N+16, H] rows ordered [cost features (N) | stock features (N) | embedding (16)],
    b1 [H], W2 [H, N], b2 [N], E [R, 16].
    """

    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    E: np.ndarray
    H: int = HIDDEN

    def as_float(self):
        return {k: bf16_to_f32(getattr(self, k)) for k in ("W1", "b1", "W2", "b2", "E")}


@dataclass
class Policy:
    """Policy selector plus its parameters.  kind: greedy | dual | mlp | gumbel."""

    kind: str
    mlp: Optional[MLPParams] = None
    seed: int = 0
    traj: int = 0


def f32_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP32 to BF16 (nearest, ties to even); returns uint16 bit patterns."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rnd = ((b >> 16) & 1) + 0x7FFF
    return ((b + rnd) >> 16).astype(np.uint16)


def bf16_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.ascontiguousarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def zipf_probs(K: int, s: float = 1.1) -> np.ndarray:
    w = np.arange(1, K + 1, dtype=np.float64) ** (-s)
    return w / w.sum()


def _orders(rng, T, K, R, s=1.1):
    p = zipf_probs(K, s)
    prod = rng.choice(K, size=T, p=p).astype(np.int32)
    reg = rng.integers(0, R, size=T, dtype=np.int64).astype(np.int32)
    return prod, reg, p


def make_instance(T, N, K, R, seed=0, stock="poisson", stock_hi=20, fill=1.05,
                  with_lam=False, lam_hi=30, cost_lo=1, cost_hi=100, zipf_s=1.1,
                  shared_tables=None) -> Instance:
    """Generic seeded FO instance.

    stock='uniform': x0 ~ U{0..stock_hi}.  stock='poisson': x0[k, n] ~
    Poisson(fill * T * p_k / N), i.e. network stock of about fill x expected
    demand, spread evenly over warehouses, so that popular products stock out at
    some warehouses.  shared_tables=(cost, lam) reuses existing tables.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    prod, reg, p = _orders(rng, T, K, R, zipf_s)
    if stock == "uniform":
        x0 = rng.integers(0, stock_hi + 1, size=(K, N), dtype=np.int64).astype(np.int32)
    elif stock == "poisson":
        mean = fill * T * p / N
        x0 = rng.poisson(np.repeat(mean[:, None], N, axis=1)).astype(np.int32)
    else:
        raise ValueError(stock)
    if shared_tables is not None:
        cost, lam = shared_tables
    else:
        cost = rng.integers(cost_lo, cost_hi + 1, size=(R, N), dtype=np.int64).astype(np.int32)
        lam = (rng.integers(0, lam_hi + 1, size=(K, N), dtype=np.int64).astype(np.int32)
               if with_lam else None)
    return Instance(T, N, K, R, np.ascontiguousarray(prod), np.ascontiguousarray(reg),
                    np.ascontiguousarray(x0), np.ascontiguousarray(cost),
                    None if lam is None else np.ascontiguousarray(lam))


def make_mlp(N: int, R: int, seed=0, H=HIDDEN, std=0.02) -> MLPParams:
    """BF16 N(0, std) parameters drawn in the fixed order W1, b1, W2, b2, E."""
    rng = np.random.Generator(np.random.PCG64(seed + 0x5EED))
    IN = 2 * N + EMB
    W1 = f32_to_bf16(rng.normal(0, std, size=(IN, H)).astype(np.float32))
    b1 = f32_to_bf16(rng.normal(0, std, size=(H,)).astype(np.float32))
    W2 = f32_to_bf16(rng.normal(0, std, size=(H, N)).astype(np.float32))
    b2 = f32_to_bf16(rng.normal(0, std, size=(N,)).astype(np.float32))
    E = f32_to_bf16(rng.normal(0, std, size=(R, EMB)).astype(np.float32))
    return MLPParams(W1, b1, W2, b2, E, H)


# ----------------------------------------------------------------------------- named workloads
def greedy_small(seed=0, T=4096):
    return make_instance(T, 8, 16, 32, seed=seed, stock="uniform", stock_hi=20)


def dual_large(seed=0, T=1 << 20, N=64, K=10_000, R=1_000):
    return make_instance(T, N, K, R, seed=seed, stock="poisson", with_lam=True)


def mlp_medium(seed=0, T=1 << 18, N=64, K=2_000, R=500):
    inst = make_instance(T, N, K, R, seed=seed, stock="poisson")
    return inst, make_mlp(N, R, seed=seed)


def batch_uneven(seed=0, B=512, Tlo=16_384, Thi=262_144, N=32, K=2_000, R=200):
    """B trajectories with their own orders and stock; shared cost table and MLP.

    Returns (instances, policies): even index greedy, odd index MLP argmax.
    """
    rng = np.random.Generator(np.random.PCG64(seed + 0xBA7C))
    Ts = rng.integers(Tlo, Thi + 1, size=B, dtype=np.int64)
    cost = rng.integers(1, 101, size=(R, N), dtype=np.int64).astype(np.int32)
    mlp = make_mlp(N, R, seed=seed)
    insts, pols = [], []
    for b in range(B):
        insts.append(make_instance(int(Ts[b]), N, K, R, seed=seed * 1_000_003 + b + 1,
                                   stock="poisson", shared_tables=(cost, None)))
        pols.append(Policy("greedy") if b % 2 == 0 else Policy("mlp", mlp=mlp))
    return insts, pols


def node_capacity(T, N, seed=0, frac=0.8, sigma=0.5):
    """Node capacity for about frac x T orders in total, spread over nodes pro
    rata to seeded log-normal(0, sigma) weights (the stand-in for the paper's
    population weights, Appendix A.3)."""
    rng = np.random.Generator(np.random.PCG64(seed + 0xCA9))
    w = rng.lognormal(0.0, sigma, size=N)
    return np.floor(frac * T * w / w.sum()).astype(np.int32)


def uniform_assignment(T, P, seed=0):
    """Each order's process drawn uniformly from 0..P-1, seeded (the uniform
    partition of Sec. 4.1, Table 1)."""
    rng = np.random.Generator(np.random.PCG64(seed + 0xA55))
    return rng.integers(0, P, size=T).astype(np.int32)


def capacity_large(seed=0, T=1 << 20, N=64, K=10_000, R=1_000, frac=0.8):
    """dual_large's orders, stock, costs and prices plus node capacity for 80%
    of the orders (the paper's FO model with capacity, Sec. 3)."""
    inst = dual_large(seed, T=T, N=N, K=K, R=R)
    inst.cap = node_capacity(T, N, seed=seed, frac=frac)
    return inst


def pg_large(seed=0, B=64, T=1 << 20, N=64, K=10_000, R=1_000):
    """B trajectories (own orders and stock, shared cost table) + one MLP."""
    rng = np.random.Generator(np.random.PCG64(seed + 0x9C))
    cost = rng.integers(1, 101, size=(R, N), dtype=np.int64).astype(np.int32)
    mlp = make_mlp(N, R, seed=seed)
    insts = [make_instance(T, N, K, R, seed=seed * 1_000_003 + b + 1, stock="poisson",
                           shared_tables=(cost, None)) for b in range(B)]
    return insts, mlp


# --------------------------------------------------------------------------- OWMR
@dataclass
class OwmrInstance:
    """One OWMR trajectory's inputs (host numpy arrays, C-contiguous)."""

    T: int
    N: int
    ret: np.ndarray  # int32 [T] retailer n(w_t) of step t
    dem: np.ndarray  # int32 [T] demand d(w_t) >= 0
    ex: np.ndarray  # int32 [T] steps since the store's previous demand (t + 1 at its first),
    #                 capped at 32,767: the demand history the retailer network sees
    cap: np.ndarray  # int32 [N] retailer capacity c_n
    x0r: np.ndarray  # int32 [N] initial retailer inventory
    sl: np.ndarray  # int32 [N] retailer reorder point s_n
    Sl: np.ndarray  # int32 [N] retailer order-up-to level S_n <= c_n
    X0: int  # initial central inventory
    s: int  # central reorder point
    S: int  # central order-up-to level


@dataclass
class OwmrNet:
    """Two-hidden-layer network (3 -> H -> H -> 1), BF16 bit patterns (uint16);
    weight matrices input-major: W1 [3, H], W2 [H, H] (row = input unit)."""

    H: int
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    w3: np.ndarray
    b3: np.ndarray


def owmr_store_weights(N, a=0.0):
    """Store-selection probabilities p_n proportional to (1 - a)^n (Appendix B.3
    ablation; a = 0 is uniform)."""
    w = (1.0 - a) ** np.arange(N, dtype=np.float64)
    return w / w.sum()


def make_owmr(T, N, seed=0, a=0.0, demand="unit", s_loc=10, S_loc=20, cap=24, s=None, S=None,
              X0=None, x0r=None):
    """Seeded OWMR instance: T steps, store of step t drawn with
    owmr_store_weights(N, a); demand 1 per step ("unit") or U{0..3} ("small");
    per-store (s_n, S_n, c_n) scalars or arrays; central (s, S) default
    (1,000, 1,000 + T / 52) so that the central warehouse replenishes about 52
    times over the horizon."""
    rng = np.random.Generator(np.random.PCG64(seed + 0x0A3B))
    p = owmr_store_weights(N, a)
    ret = rng.choice(N, size=T, p=p).astype(np.int32)
    if demand == "unit":
        dem = np.ones(T, np.int32)
    elif demand == "small":
        dem = rng.integers(0, 4, size=T).astype(np.int32)
    else:
        raise ValueError(demand)
    full = lambda v: np.ascontiguousarray(np.broadcast_to(np.asarray(v, np.int32), (N,)))
    capa, sla, Sla = full(cap), full(s_loc), full(S_loc)
    s = 1_000 if s is None else int(s)
    S = s + max(1, T // 52) if S is None else int(S)
    X0 = S if X0 is None else int(X0)
    x0r = Sla.copy() if x0r is None else full(x0r)
    return OwmrInstance(T, N, ret, dem, demand_gaps(ret), capa, x0r, sla, Sla, X0, s, S)


def demand_gaps(ret):
    """Per step, the steps since the same store's previous demand (t + 1 for its
    first), capped at 32,767."""
    T = len(ret)
    t = np.arange(T, dtype=np.int64)
    order = np.lexsort((t, ret))
    rs, ts = ret[order], t[order]
    prev = np.full(T, -1, np.int64)
    if T > 1:
        same = rs[1:] == rs[:-1]
        prev[1:][same] = ts[:-1][same]
    gap = np.empty(T, np.int64)
    gap[order] = ts - prev
    return np.minimum(gap, 32_767).astype(np.int32)


def make_owmr_net(H=512, seed=0, std=0.02) -> OwmrNet:
    """BF16 N(0, std) parameters drawn in the order W1, b1, W2, b2, w3, b3."""
    rng = np.random.Generator(np.random.PCG64(seed + 0x0E7))
    g = lambda *shape: f32_to_bf16(rng.normal(0.0, std, size=shape).astype(np.float32))
    W1, b1, W2, b2, w3, b3 = g(3, H), g(H), g(H, H), g(H), g(H), g(1)
    return OwmrNet(H, W1, b1, W2, b2, w3, b3)


def owmr_base(seed=0, T=3_650_000, N=4_000, a=0.0, H=512):
    """Appendix B.3's base case: 10,000 unit demands a day for a year over
    4,000 stores, stores (s_n, S_n) = (10, 20) with capacity 24, central
    (s, S) = (1,000, 71,000) (about one replenishment a week), width-512
    network."""
    inst = make_owmr(T, N, seed=seed, a=a, s=1_000, S=71_000)
    return inst, make_owmr_net(H, seed=seed)
