"""GPU parity of Algorithm 1 under the product partition of Sec. 3 (processor
of product k: k mod P), greedy and bid-price policies, with and without node
capacity, against the CPU oracle's Algorithm 1 for the same assignment of
orders to processes.  Every iterate, the pass count, the path, its cost and the
final stock are compared bit for bit; Theorem 3.1 bounds the passes."""
import numpy as np
import pytest

import oracle
import paper_2406_01939_b300 as pic
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.session import DeviceInstance
from paper_2406_01939_b300.synth import Policy

pytestmark = pytest.mark.gpu


def make(seed, T, N, K, cap_frac=None, R=7, fill=0.9):
    inst = synth.make_instance(T, N, K, R, seed=seed, stock="poisson", fill=fill, with_lam=True)
    if cap_frac is not None:
        inst.cap = synth.node_capacity(T, N, seed=seed, frac=cap_frac)
    return inst


def proc_of(inst, P):
    return (inst.prod % P).astype(np.int32)


def check(inst, kind, P, dev=None, **kw):
    pol = Policy(kind)
    seq = oracle.seq_sim(inst, pol)
    want = oracle.picard_partition(inst, pol, proc_of(inst, P), **kw)
    d = dev or DeviceInstance(inst)
    got = d.simulate(pol, "products", num_chunks=P, **kw)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
    assert got["iters"] == want["iters"], (kind, P, got["iters"], want["iters"])
    assert got["total_cost"] == seq["total_cost"] and got["lost"] == seq["lost"]
    np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])
    assert got["num_chunks"] == min(P, inst.K)
    return got, want, seq


@pytest.mark.parametrize("N", [5, 32, 33, 64, 100, 127])
def test_random_shapes_bit_exact(N):
    """Ragged lane counts, 1 to K (and more than K) processors, both policies,
    binding capacity, ample capacity and none."""
    rng = np.random.default_rng(N)
    for trial in range(3):
        T = int(rng.integers(200, 2500))
        K = int(rng.integers(2, 30))
        frac = [None, float(rng.uniform(0.3, 0.9)), 1.5][trial]
        inst = make(50 * N + trial, T, N, K, frac)
        d = DeviceInstance(inst)
        for kind in ("greedy", "dual"):
            for P in sorted({1, 3, K, K + 4}):
                check(inst, kind, P, dev=d)


def test_every_iterate_matches_algorithm_1():
    """Capping the passes at k returns alpha^k of Algorithm 1 under the product
    partition, for every k, with the status NOT_CONVERGED before the last."""
    inst = make(7, 1500, 24, 16, cap_frac=0.5)
    d = DeviceInstance(inst)
    for kind in ("greedy", "dual"):
        for P in (4, 16):
            want = oracle.picard_partition(inst, Policy(kind), proc_of(inst, P), record=True)
            assert want["iters"] >= 3
            for k in range(1, want["iters"] + 1):
                got = d.simulate(Policy(kind), "products", num_chunks=P, max_iters=k,
                                 raise_on_error=False)
                assert got["status"] == (pic.PIC_OK if k == want["iters"] else pic.PIC_ERR_NOT_CONVERGED)
                np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["iterates"][k - 1])


def test_theorem_3_1_pass_bound():
    """Thm. 3.1: with a bid-price (or, inventory not binding, greedy) policy the
    product-partitioned cache is exact after at most |Q_T| + 1 passes, Q_T the
    nodes whose capacity the sequential path exhausts; one more confirms it."""
    rng = np.random.default_rng(31)
    for trial in range(6):
        T = int(rng.integers(500, 4000))
        N, K = int(rng.integers(4, 40)), int(rng.integers(3, 40))
        inst = make(300 + trial, T, N, K, float(rng.uniform(0.2, 1.0)))
        d = DeviceInstance(inst)
        seq = oracle.seq_sim(inst, Policy("dual"))
        Q = int((seq["c_final"] == 0).sum())
        for P in (2, K):
            got = d.simulate(Policy("dual"), "products", num_chunks=P)
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
            assert got["iters"] <= Q + 2, (got["iters"], Q)
        if trial % 2 == 0:
            inst.x0 = np.full((K, N), T, np.int32)  # inventory not binding: greedy as well
            gs = oracle.seq_sim(inst, Policy("greedy"))
            Qg = int((gs["c_final"] == 0).sum())
            got = DeviceInstance(inst).simulate(Policy("greedy"), "products", num_chunks=K)
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), gs["actions"])
            assert got["iters"] <= Qg + 2


def test_without_capacity_two_passes():
    """No capacity: every processor owns its products' inventory outright, so
    pass 1 is exact and pass 2 confirms it."""
    inst = make(8, 3000, 40, 25)
    d = DeviceInstance(inst)
    for kind in ("greedy", "dual"):
        for P in (1, 5, 25):
            got, want, _ = check(inst, kind, P, dev=d)
            assert got["iters"] == 2


def test_warm_start():
    inst = make(9, 2500, 16, 12, cap_frac=0.6)
    d = DeviceInstance(inst)
    pol = Policy("dual")
    seq = oracle.seq_sim(inst, pol)["actions"]
    assert d.simulate(pol, "products", num_chunks=6, alpha_init=seq)["iters"] == 1
    rng = np.random.default_rng(0)
    init = rng.integers(-1, inst.N, inst.T).astype(np.int8)
    want = oracle.picard_partition(inst, pol, proc_of(inst, 6), alpha_init=init)
    got = d.simulate(pol, "products", num_chunks=6, alpha_init=init)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq)
    assert got["iters"] == want["iters"]


def test_degenerate_instances():
    """T = 0, zero capacity at every node, one order, one product."""
    for T, N, K, frac in ((0, 4, 3, 0.5), (1, 3, 1, 0.5), (400, 6, 1, 0.4), (500, 9, 7, 0.0)):
        inst = make(T + N, T, N, K, frac)
        if frac == 0.0:
            inst.cap = np.zeros(N, np.int32)
        d = DeviceInstance(inst)
        for kind in ("greedy", "dual"):
            got = d.simulate(Policy(kind), "products", num_chunks=2)
            seq = oracle.seq_sim(inst, Policy(kind))
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
            np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])
            if T:
                want = oracle.picard_partition(inst, Policy(kind), proc_of(inst, 2))
                assert got["iters"] == want["iters"]
            else:
                assert got["iters"] == 1


def test_invalid_inputs():
    inst = make(5, 300, 8, 5, cap_frac=0.5)
    d = DeviceInstance(inst)
    with pytest.raises(pic.PicError) as e:
        d.simulate(Policy("greedy"), "products", alpha_init=np.full(inst.T, inst.N, np.int8))
    assert e.value.status == pic.PIC_ERR_INVALID_ARG
    plain = make(5, 300, 8, 5)
    mlp = synth.make_mlp(plain.N, plain.R, seed=1)
    with pytest.raises(pic.PicError) as e:
        DeviceInstance(plain).simulate(Policy("mlp", mlp=mlp), "products")
    assert e.value.status == pic.PIC_ERR_UNSUPPORTED
    with pytest.raises(pic.PicError) as e:
        DeviceInstance(plain).simulate(Policy("greedy"), "products", max_steps=64)
    assert e.value.status == pic.PIC_ERR_UNSUPPORTED


def test_full_size_capacity_workload():
    """T = 2^20, N = 64, K = 10,000, R = 1,000, capacity for 80% of the orders,
    bid-price policy, one processor per product: the oracle's sequential path,
    cost and final stock, within Theorem 3.1's pass bound."""
    inst = synth.capacity_large(0)
    pol = Policy("dual")
    seq = oracle.seq_sim(inst, pol)
    Q = int((seq["c_final"] == 0).sum())
    got = DeviceInstance(inst).simulate(pol, "products")
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
    assert got["total_cost"] == seq["total_cost"] and got["lost"] == seq["lost"]
    np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])
    assert got["iters"] <= Q + 2
