"""GPU parity of the FO model with node capacity (Sec. 3 state (x, c); greedy
and bid-price policies) against the CPU oracle, through the C ABI.  Integer
outputs are compared bit for bit; the pass count of Algorithm 1 on contiguous
chunks must equal the oracle's."""
import numpy as np
import pytest
import torch

import oracle
import paper_2406_01939_b300 as pic
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.session import DeviceBatch, DeviceInstance
from paper_2406_01939_b300.synth import Instance, Policy

pytestmark = pytest.mark.gpu


def cap_inst(seed, T, N, K, R=7, frac=0.7, fill=0.9):
    inst = synth.make_instance(T, N, K, R, seed=seed, stock="poisson", fill=fill, with_lam=True)
    inst.cap = synth.node_capacity(T, N, seed=seed, frac=frac)
    return inst


def check(inst, kind, M, dev=None, **kw):
    pol = Policy(kind)
    seq = oracle.seq_sim(inst, pol)
    want = oracle.picard_chunked(inst, pol, M)
    d = dev or DeviceInstance(inst)
    got = d.simulate(pol, "picard", num_chunks=M, **kw)
    a = got["actions"].cpu().numpy()
    np.testing.assert_array_equal(a, seq["actions"])
    assert got["iters"] == want["iters"], (got["iters"], want["iters"])
    assert got["total_cost"] == seq["total_cost"] and got["lost"] == seq["lost"]
    np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])
    assert got["num_chunks"] == M
    return got, want


@pytest.mark.parametrize("N", [5, 32, 33, 64, 100])
def test_capacity_random_shapes_bit_exact(N):
    """Ragged lane counts (N = 5, 33, 100), several chunk lengths up to 64,
    both policies: path, cost, a^phi count, final stock, passes."""
    rng = np.random.default_rng(N)
    for trial in range(3):
        T = int(rng.integers(300, 3000))
        inst = cap_inst(100 * N + trial, T, N, int(rng.integers(2, 40)), frac=float(rng.uniform(0.3, 1.1)))
        d = DeviceInstance(inst)
        for kind in ("greedy", "dual"):
            for L in (64, 37, 8, 1):
                check(inst, kind, -(-T // L), dev=d)


def test_capacity_every_iterate_matches_algorithm_1():
    """Capping the passes at k returns alpha^k of Algorithm 1 (contiguous
    chunks with capacity), for every k."""
    inst = cap_inst(7, 2000, 24, 12, frac=0.6)
    pol = Policy("dual")
    M = -(-inst.T // 50)
    want = oracle.picard_partition(inst, pol, np.arange(inst.T) // 50, record=True)
    assert want["iters"] == oracle.picard_chunked(inst, pol, M)["iters"]
    d = DeviceInstance(inst)
    for k in range(1, want["iters"] + 1):
        got = d.simulate(pol, "picard", num_chunks=M, max_iters=k, raise_on_error=False)
        assert got["status"] == (pic.PIC_OK if k == want["iters"] else pic.PIC_ERR_NOT_CONVERGED)
        np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["iterates"][k - 1])


def test_capacity_sequential_mode_bit_exact():
    for seed, N in ((1, 8), (2, 64), (3, 77)):
        inst = cap_inst(seed, 5000, N, 30, frac=0.5)
        d = DeviceInstance(inst)
        for kind in ("greedy", "dual"):
            seq = oracle.seq_sim(inst, Policy(kind))
            got = d.simulate(Policy(kind), "sequential")
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
            np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])
            assert got["total_cost"] == seq["total_cost"] and got["lost"] == seq["lost"]


def test_ample_capacity_equals_inventory_only_path():
    """Capacity that cannot bind gives the inventory-only path of the same
    instance (a different kernel)."""
    inst = cap_inst(4, 4000, 40, 25)
    inst.cap = np.full(inst.N, inst.T, np.int32)
    base = Instance(inst.T, inst.N, inst.K, inst.R, inst.prod, inst.reg, inst.x0, inst.cost, inst.lam)
    a = DeviceInstance(inst).simulate(Policy("dual"), "picard", num_chunks=100)
    b = DeviceInstance(base).simulate(Policy("dual"), "picard", num_chunks=100)
    assert torch.equal(a["actions"], b["actions"]) and a["total_cost"] == b["total_cost"]
    assert torch.equal(a["final_stock"], b["final_stock"])


def test_zero_capacity_and_tiny_instances():
    inst = cap_inst(5, 700, 6, 4)
    inst.cap = np.zeros(6, np.int32)
    got = DeviceInstance(inst).simulate(Policy("greedy"), "picard", num_chunks=20)
    assert (got["actions"].cpu().numpy() == -1).all() and got["iters"] == 1
    assert got["lost"] == 700 and got["total_cost"] == 0
    for T in (1, 2, 63, 64, 65):
        inst = cap_inst(T, T, 3, 2, frac=0.5)
        for M in sorted({-(-T // 64), T}):
            check(inst, "greedy", M)


def test_capacity_warm_start():
    """A cache started from another path still reaches the sequential path; with
    the sequential path itself as alpha_init, one confirming pass."""
    inst = cap_inst(9, 3000, 16, 20, frac=0.6)
    pol = Policy("dual")
    seq = oracle.seq_sim(inst, pol)["actions"]
    d = DeviceInstance(inst)
    M = -(-inst.T // 64)
    rng = np.random.default_rng(0)
    init = rng.integers(-1, inst.N, inst.T).astype(np.int8)
    want = oracle.picard_chunked(inst, pol, M, alpha_init=init)
    got = d.simulate(pol, "picard", num_chunks=M, alpha_init=init)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq)
    assert got["iters"] == want["iters"]
    again = d.simulate(pol, "picard", num_chunks=M, alpha_init=seq)
    assert again["iters"] == 1


def test_capacity_invalid_inputs():
    inst = cap_inst(6, 1000, 8, 5)
    d = DeviceInstance(inst)
    with pytest.raises(pic.PicError) as e:
        d.simulate(Policy("greedy"), "picard", num_chunks=10)  # chunks of 100 orders
    assert e.value.status == pic.PIC_ERR_INVALID_ARG and "64" in str(e.value)
    mlp = synth.make_mlp(inst.N, inst.R, seed=1)
    with pytest.raises(pic.PicError) as e:
        d.simulate(Policy("mlp", mlp=mlp), "picard")
    assert e.value.status == pic.PIC_ERR_UNSUPPORTED
    bad = cap_inst(6, 1000, 8, 5)
    bad.cap = bad.cap.copy()
    bad.cap[3] = -2
    with pytest.raises(pic.PicError) as e:
        DeviceInstance(bad)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG and "cap" in str(e.value)
    with pytest.raises(pic.PicError) as e:
        DeviceBatch([inst, cap_inst(7, 500, 8, 5)])
    assert e.value.status == pic.PIC_ERR_UNSUPPORTED


def test_capacity_large_full_size():
    """T = 2^20, N = 64, K = 10,000, R = 1,000, capacity for 80% of the orders,
    bid-price policy, chunks of 64 orders: the oracle's sequential path and its
    pass count; the GPU sequential simulator agrees."""
    inst = synth.capacity_large(0)
    pol = Policy("dual")
    M = inst.T // 64
    seq = oracle.seq_sim(inst, pol)
    want = oracle.picard_chunked(inst, pol, M)
    d = DeviceInstance(inst)
    got = d.simulate(pol, "picard", num_chunks=M)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
    np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])
    assert got["iters"] == want["iters"]
    assert got["total_cost"] == seq["total_cost"] and got["lost"] == seq["lost"]
    s = d.simulate(pol, "sequential")
    assert torch.equal(s["actions"], got["actions"])
