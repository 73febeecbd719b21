"""Pins for the oracle's FO model with node capacity (Sec. 3: state (x, c), an
order may go to node n only if x[k][n] > 0 and c[n] > 0) and for Algorithm 1
under arbitrary assignments of time-steps to processes.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.synth import Instance, Policy


def tiny_cap(rng, T=None, N=None, K=None, R=None, xmax=4, capmax=6, lam=True):
    T = int(rng.integers(0, 41)) if T is None else T
    N = int(rng.integers(1, 6)) if N is None else N
    K = int(rng.integers(1, 5)) if K is None else K
    R = int(rng.integers(1, 4)) if R is None else R
    inst = Instance(
        T, N, K, R,
        rng.integers(0, K, T).astype(np.int32), rng.integers(0, R, T).astype(np.int32),
        rng.integers(0, xmax + 1, (K, N)).astype(np.int32),
        rng.integers(1, 6, (R, N)).astype(np.int32),
        rng.integers(0, 4, (K, N)).astype(np.int32) if lam else None)
    inst.cap = rng.integers(0, capmax + 1, N).astype(np.int32)
    return inst


def replay(inst, actions):
    """(stock rows, capacity vectors) seen before every t under an action path."""
    x = inst.x0.astype(np.int64).copy()
    c = inst.cap.astype(np.int64).copy()
    rows, caps = [], []
    for t in range(inst.T):
        k = inst.prod[t]
        rows.append(x[k].copy())
        caps.append(c.copy())
        a = actions[t]
        if a >= 0:
            x[k, a] -= 1
            c[a] -= 1
    return rows, caps, x, c


def first_exact(iterates, seq):
    for k, a in enumerate(iterates, 1):
        if np.array_equal(a, seq):
            return k
    return None


def contiguous(T, M):
    L = -(-T // M) if T else 1
    return (np.arange(T) // L).astype(np.int32)


# ----------------------------------------------------------------------------- sequential
def test_cap_seq_textbook_argmin_every_step():
    """Each action is the textbook arg min (lowest index on ties) of the policy's
    score over {n : x[k][n] > 0, c[n] > 0}, a^phi iff that set is empty; stock
    and capacity never go negative; shipped units add up per product and per
    node; cost is the sum over fulfilled orders."""
    rng = np.random.default_rng(11)
    for trial in range(200):
        inst = tiny_cap(rng)
        for kind in ("greedy", "dual"):
            out = oracle.seq_sim(inst, Policy(kind))
            a = out["actions"]
            rows, caps, xf, cf = replay(inst, a)
            cost = 0
            for t in range(inst.T):
                k, r = inst.prod[t], inst.reg[t]
                feas = [n for n in range(inst.N) if rows[t][n] > 0 and caps[t][n] > 0]
                score = lambda n: inst.cost[r, n] - (inst.lam[k, n] if kind == "dual" else 0)
                want = min(feas, key=lambda n: (score(n), n)) if feas else -1
                assert a[t] == want, (trial, kind, t)
                if a[t] >= 0:
                    cost += int(inst.cost[r, a[t]])
            assert (xf >= 0).all() and (cf >= 0).all()
            np.testing.assert_array_equal(out["x_final"], xf)
            np.testing.assert_array_equal(out["c_final"], cf)
            shipped = np.bincount(a[a >= 0], minlength=inst.N)
            np.testing.assert_array_equal(inst.cap - out["c_final"], shipped)
            assert out["total_cost"] == cost and out["lost"] == int((a < 0).sum())


def test_cap_ample_capacity_is_inventory_only_model():
    """Capacity that can never bind (c_1 >= T at every node) leaves the
    inventory-only dynamics: same path, and the same Picard iterates."""
    rng = np.random.default_rng(12)
    for trial in range(60):
        inst = tiny_cap(rng, T=int(rng.integers(1, 60)))
        inst.cap = np.full(inst.N, inst.T, np.int32)
        base = Instance(inst.T, inst.N, inst.K, inst.R, inst.prod, inst.reg, inst.x0, inst.cost,
                        inst.lam)
        for kind in ("greedy", "dual"):
            pol = Policy(kind)
            np.testing.assert_array_equal(oracle.seq_sim(inst, pol)["actions"],
                                          oracle.seq_sim(base, pol)["actions"])
            M = int(rng.integers(1, 8))
            a = oracle.picard_chunked(inst, pol, M, record=True)
            b = oracle.picard_chunked(base, pol, M, record=True)
            assert a["iters"] == b["iters"]
            np.testing.assert_array_equal(a["iterates"], b["iterates"])


def test_cap_zero_capacity_loses_everything():
    inst = synth.make_instance(300, 5, 4, 3, seed=2, with_lam=True)
    inst.cap = np.zeros(5, np.int32)
    out = oracle.seq_sim(inst, Policy("dual"))
    assert (out["actions"] == -1).all() and out["total_cost"] == 0 and out["lost"] == 300
    r = oracle.picard_chunked(inst, Policy("dual"), 7)
    assert r["iters"] == 1 and (r["actions"] == -1).all()  # the all-a^phi cache is the fixed point


def test_cap_single_node_closed_form():
    """One node, one product: the first min(x0, c_1) orders are fulfilled."""
    for x0, c1, T in [(5, 3, 10), (3, 5, 10), (0, 4, 6), (7, 7, 7), (9, 2, 4)]:
        inst = Instance(T, 1, 1, 1, np.zeros(T, np.int32), np.zeros(T, np.int32),
                        np.array([[x0]], np.int32), np.array([[4]], np.int32))
        inst.cap = np.array([c1], np.int32)
        a = oracle.seq_sim(inst, Policy("greedy"))["actions"]
        m = min(x0, c1, T)
        assert (a[:m] == 0).all() and (a[m:] == -1).all()


# ----------------------------------------------------------------------------- Algorithm 1
def test_partition_contiguous_equals_literal_without_capacity():
    """picard_partition with proc[t] = t // L is Algorithm 1 on contiguous blocks:
    iterate for iterate the oracle's picard_literal, for every policy kind."""
    rng = np.random.default_rng(13)
    for trial in range(40):
        inst = tiny_cap(rng, T=int(rng.integers(1, 40)))
        inst.cap = None
        mlp = synth.make_mlp(inst.N, inst.R, seed=trial)
        for pol in (Policy("greedy"), Policy("dual"), Policy("mlp", mlp=mlp),
                    Policy("gumbel", mlp=mlp, seed=trial, traj=1)):
            M = int(rng.integers(1, inst.T + 1))
            proc = contiguous(inst.T, M)
            a = oracle.picard_partition(inst, pol, proc, record=True)
            b = oracle.picard_literal(inst, pol, int(proc.max()) + 1, max_iters=inst.T + 1,
                                      record=True)
            assert a["iters"] == b["iters"]
            np.testing.assert_array_equal(a["iterates"], b["iterates"])


def test_exhaustive_tiny_capacity_literal_equals_chunked_and_seq():
    """Exhaustive family: T = 5 orders, N = 2 nodes, K = 2 products, x0 in
    {0,1,2}^4, c_1 in {0,1,2,3}^2, every product sequence; every M = 1..5.  The
    closed-form block prefix (c = max(0, c_1 - q)) gives Algorithm 1's iterates,
    and the fixed point is the sequential path (Prop. 1)."""
    T, N, K = 5, 2, 2
    cost = np.array([[3, 1], [1, 3]], np.int32)
    reg = np.array([0, 1, 0, 0, 1], np.int32)
    count = 0
    for x0f in itertools.product(range(3), repeat=K * N):
        for capv in itertools.product(range(4), repeat=N):
            for prodv in itertools.product(range(K), repeat=T):
                if (sum(prodv) + sum(x0f) + sum(capv)) % 5:  # a fifth of the family
                    continue
                inst = Instance(T, N, K, 2, np.array(prodv, np.int32), reg,
                                np.array(x0f, np.int32).reshape(K, N), cost)
                inst.cap = np.array(capv, np.int32)
                pol = Policy("greedy")
                seq = oracle.seq_sim(inst, pol)["actions"]
                for M in range(1, T + 1):
                    lit = oracle.picard_partition(inst, pol, contiguous(T, M), record=True)
                    ch = oracle.picard_chunked(inst, pol, M, max_iters=T + 1, record=True)
                    assert lit["iters"] == ch["iters"]
                    np.testing.assert_array_equal(lit["iterates"], ch["iterates"])
                    np.testing.assert_array_equal(ch["actions"], seq)
                count += 1
    assert count > 1000


def test_prop1_any_partition_reaches_seq():
    """Prop. 1: for contiguous blocks, product partitions and a uniform random
    assignment alike, the fixed point is the sequential path, within T passes."""
    rng = np.random.default_rng(14)
    for trial in range(60):
        inst = tiny_cap(rng, T=int(rng.integers(1, 40)))
        for kind in ("greedy", "dual"):
            pol = Policy(kind)
            seq = oracle.seq_sim(inst, pol)["actions"]
            M = int(rng.integers(1, 6))
            for proc in (contiguous(inst.T, M), rng.integers(0, M, inst.K)[inst.prod],
                         rng.integers(0, M, inst.T)):
                out = oracle.picard_partition(inst, pol, np.asarray(proc, np.int32))
                assert out["converged"] and out["iters"] <= inst.T + 1
                np.testing.assert_array_equal(out["actions"], seq)


def _product_partition_case(seed, ample_stock):
    rng = np.random.default_rng(seed)
    T = int(rng.integers(200, 1200))
    N = int(rng.integers(2, 9))
    K = int(rng.integers(2, 30))
    inst = synth.make_instance(T, N, K, 7, seed=seed, stock="poisson",
                               fill=float(rng.uniform(0.5, 1.5)), with_lam=True)
    if ample_stock:
        inst.x0 = np.full((K, N), T, np.int32)
    inst.cap = synth.node_capacity(T, N, seed=seed, frac=float(rng.uniform(0.3, 1.2)))
    M = int(rng.integers(2, 12))
    proc = rng.integers(0, M, size=K)[inst.prod].astype(np.int32)
    return inst, proc


@pytest.mark.parametrize("seed", range(8))
def test_thm31_special_case_greedy_ample_inventory(seed):
    """Sec. 3.1 special case: inventory not a constraint, greedy policy, product
    partitions.  The cache is exact after at most |Q_T| + 1 passes, Q_T the nodes
    whose capacity the sequential path exhausts."""
    inst, proc = _product_partition_case(2 * seed, True)
    pol = Policy("greedy")
    seq = oracle.seq_sim(inst, pol)
    Q = int((seq["c_final"] == 0).sum())
    out = oracle.picard_partition(inst, pol, proc, record=True)
    k = first_exact(out["iterates"], seq["actions"])
    assert k is not None and k <= Q + 1
    assert out["iters"] == k + (0 if k == 1 and out["iters"] == 1 else 1)


@pytest.mark.parametrize("seed", range(8))
def test_thm31_bid_price_with_inventory(seed):
    """Thm. 3.1: a bid-price policy meets Assumptions 1-3, so with inventory
    constraints and product partitions the cache is exact after at most
    |Q_T| + 1 passes."""
    inst, proc = _product_partition_case(2 * seed + 1, False)
    pol = Policy("dual")
    seq = oracle.seq_sim(inst, pol)
    Q = int((seq["c_final"] == 0).sum())
    out = oracle.picard_partition(inst, pol, proc, record=True)
    k = first_exact(out["iterates"], seq["actions"])
    assert k is not None and k <= Q + 1


def test_product_partitions_without_binding_capacity_one_pass():
    """With Q_T empty (capacity never binds) product partitions are exact after
    one pass: every process owns its products' inventory outright."""
    rng = np.random.default_rng(15)
    for trial in range(20):
        inst = tiny_cap(rng, T=int(rng.integers(1, 60)))
        inst.cap = np.full(inst.N, inst.T, np.int32)
        M = int(rng.integers(1, 5))
        proc = rng.integers(0, M, inst.K)[inst.prod].astype(np.int32)
        for kind in ("greedy", "dual"):
            out = oracle.picard_partition(inst, Policy(kind), proc, record=True)
            np.testing.assert_array_equal(out["iterates"][0], oracle.seq_sim(inst, Policy(kind))["actions"])
            assert out["iters"] == 2


def test_capacity_rejects_mlp_and_bad_capacity():
    inst = tiny_cap(np.random.default_rng(3), T=10)
    mlp = synth.make_mlp(inst.N, inst.R, seed=1)
    with pytest.raises(ValueError):
        oracle.seq_sim(inst, Policy("mlp", mlp=mlp))
    inst.cap = inst.cap.copy()
    inst.cap[0] = -1
    with pytest.raises(ValueError):
        oracle.seq_sim(inst, Policy("greedy"))
