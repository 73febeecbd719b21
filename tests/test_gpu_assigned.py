"""GPU parity of Algorithm 1 for a caller's assignment of orders to processes
(uniform random as in Sec. 4.1 / Table 1, contiguous, by product), greedy and
bid-price policies, without and with node capacity, against the CPU oracle's
Algorithm 1 for the same assignment: every iterate, the pass count, the path,
its cost and the final stock bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2406_01939_b300 as pic
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.session import DeviceInstance
from paper_2406_01939_b300.synth import Policy

pytestmark = pytest.mark.gpu


def make(seed, T, N, K, R=7, fill=0.9):
    return synth.make_instance(T, N, K, R, seed=seed, stock="poisson", fill=fill, with_lam=True)


def check(inst, kind, proc, P, dev=None, **kw):
    pol = Policy(kind)
    seq = oracle.seq_sim(inst, pol)
    want = oracle.picard_partition(inst, pol, proc, **kw)
    d = dev or DeviceInstance(inst)
    got = d.simulate(pol, "assigned", num_chunks=P, proc=proc, **kw)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
    assert got["iters"] == want["iters"], (kind, P, got["iters"], want["iters"])
    assert got["total_cost"] == seq["total_cost"] and got["lost"] == seq["lost"]
    np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])
    assert got["num_chunks"] == P
    return got, want


@pytest.mark.parametrize("N", [5, 32, 33, 64, 100, 127])
def test_uniform_random_assignment_bit_exact(N):
    """Ragged lane counts; 1 to T processes; scarce and ample stock."""
    rng = np.random.default_rng(N)
    for trial in range(3):
        T = int(rng.integers(200, 3000))
        inst = make(70 * N + trial, T, N, int(rng.integers(2, 40)), fill=[0.9, 0.5, 3.0][trial])
        d = DeviceInstance(inst)
        for kind in ("greedy", "dual"):
            for P in sorted({1, 7, 64, T}):
                check(inst, kind, synth.uniform_assignment(T, P, seed=trial), P, dev=d)


def test_every_iterate_matches_algorithm_1():
    inst = make(3, 2000, 24, 20, fill=0.6)
    d = DeviceInstance(inst)
    for kind in ("greedy", "dual"):
        proc = synth.uniform_assignment(inst.T, 32, seed=5)
        want = oracle.picard_partition(inst, Policy(kind), proc, record=True)
        assert want["iters"] >= 3
        for k in range(1, want["iters"] + 1):
            got = d.simulate(Policy(kind), "assigned", num_chunks=32, proc=proc, max_iters=k,
                             raise_on_error=False)
            assert got["status"] == (pic.PIC_OK if k == want["iters"] else pic.PIC_ERR_NOT_CONVERGED)
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["iterates"][k - 1])


def test_contiguous_and_product_assignments():
    """proc[t] = t // L is the contiguous-chunk mode's partition and proc[t] =
    k_t mod P the product mode's: same passes, same iterates."""
    inst = make(4, 4000, 48, 30, fill=0.7)
    d = DeviceInstance(inst)
    for kind in ("greedy", "dual"):
        for M in (16, 125):
            L = -(-inst.T // M)
            proc = (np.arange(inst.T) // L).astype(np.int32)
            got, _ = check(inst, kind, proc, M, dev=d)
            assert got["iters"] == d.simulate(Policy(kind), "picard", num_chunks=M)["iters"]
        for P in (3, 30):
            proc = (inst.prod % P).astype(np.int32)
            got, _ = check(inst, kind, proc, P, dev=d)
            assert got["iters"] == d.simulate(Policy(kind), "products", num_chunks=P)["iters"]


def test_warm_start_and_degenerate():
    inst = make(9, 2500, 16, 12, fill=0.6)
    d = DeviceInstance(inst)
    pol = Policy("dual")
    seq = oracle.seq_sim(inst, pol)["actions"]
    proc = synth.uniform_assignment(inst.T, 50, seed=1)
    assert d.simulate(pol, "assigned", num_chunks=50, proc=proc, alpha_init=seq)["iters"] == 1
    init = np.random.default_rng(0).integers(-1, inst.N, inst.T).astype(np.int8)
    want = oracle.picard_partition(inst, pol, proc, alpha_init=init)
    got = d.simulate(pol, "assigned", num_chunks=50, proc=proc, alpha_init=init)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq)
    assert got["iters"] == want["iters"]
    for T, K in ((0, 3), (1, 1), (300, 1)):
        inst = make(T + 1, T, 6, K, fill=0.5)
        proc = synth.uniform_assignment(T, 4, seed=T)
        got = DeviceInstance(inst).simulate(pol, "assigned", num_chunks=4, proc=proc)
        s = oracle.seq_sim(inst, pol)
        np.testing.assert_array_equal(got["actions"].cpu().numpy(), s["actions"])
        np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), s["x_final"])
        if T:
            assert got["iters"] == oracle.picard_partition(inst, pol, proc)["iters"]


def test_invalid_inputs():
    inst = make(5, 300, 8, 5)
    d = DeviceInstance(inst)
    proc = synth.uniform_assignment(inst.T, 4, seed=0)
    bad = proc.copy()
    bad[17] = 4
    with pytest.raises(pic.PicError) as e:
        d.simulate(Policy("greedy"), "assigned", num_chunks=4, proc=bad)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG and "proc" in str(e.value)
    with pytest.raises(pic.PicError) as e:
        d.simulate(Policy("greedy"), "assigned", num_chunks=0, proc=proc)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG
    with pytest.raises(pic.PicError) as e:
        d.simulate(Policy("greedy"), "assigned", num_chunks=4)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG
    mlp = synth.make_mlp(inst.N, inst.R, seed=1)
    with pytest.raises(pic.PicError) as e:
        d.simulate(Policy("mlp", mlp=mlp), "assigned", num_chunks=4, proc=proc)
    assert e.value.status == pic.PIC_ERR_UNSUPPORTED


def test_full_size_uniform_assignment():
    """dual_large (T = 2^20, K = 10,000, Zipf 1.1) over 4,096 uniformly drawn
    processes: the oracle's sequential path, cost and final stock."""
    inst = synth.dual_large(0)
    pol = Policy("dual")
    seq = oracle.seq_sim(inst, pol)
    proc = synth.uniform_assignment(inst.T, 4096, seed=0)
    got = DeviceInstance(inst).simulate(pol, "assigned", num_chunks=4096, proc=proc)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
    assert got["total_cost"] == seq["total_cost"] and got["lost"] == seq["lost"]
    np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])


@pytest.mark.parametrize("N", [8, 33, 64])
def test_uniform_random_assignment_with_capacity(N):
    """Node capacity (the Sec. 3 state (x, c)) under uniform random assignments,
    the setting of Table 1: every process replays its own view of the horizon.
    Scarce and ample stock and capacity, 1 to 40 processes, every iterate."""
    rng = np.random.default_rng(100 + N)
    for trial in range(3):
        T = int(rng.integers(50, 1500))
        K = int(rng.integers(2, 12))
        inst = make(1000 + 10 * N + trial, T, N, K, fill=float(rng.uniform(0.4, 1.5)))
        inst.cap = synth.node_capacity(T, N, seed=trial, frac=float(rng.uniform(0.3, 0.9)))
        d = DeviceInstance(inst)
        for P in (1, 7, 40):
            proc = synth.uniform_assignment(T, P, seed=trial)
            for kind in ("greedy", "dual"):
                check(inst, kind, proc, P, dev=d)
        proc = synth.uniform_assignment(T, 9, seed=5)
        rec = oracle.picard_partition(inst, Policy("dual"), proc, record=True)
        for k in sorted({1, 2, rec["iters"]}):
            g = d.simulate(Policy("dual"), "assigned", num_chunks=9, proc=proc, max_iters=k,
                           raise_on_error=False)
            np.testing.assert_array_equal(g["actions"].cpu().numpy(), rec["iterates"][k - 1])


def test_capacity_replay_rejects_bad_processes_and_handles_empty_ones():
    """With capacity: a process outside [0, P) is an error before any pass;
    processes that own no orders (P larger than the orders) are skipped."""
    inst = make(77, 200, 16, 4, fill=0.8)
    inst.cap = synth.node_capacity(inst.T, inst.N, seed=1, frac=0.6)
    d = DeviceInstance(inst)
    proc = synth.uniform_assignment(inst.T, 5, seed=2)
    bad = proc.copy()
    bad[3] = 5
    with pytest.raises(pic.PicError) as e:
        d.simulate(Policy("dual"), "assigned", num_chunks=5, proc=bad)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG and "proc" in str(e.value)
    sparse = np.arange(inst.T, dtype=np.int32) % 7 * 50  # processes 0, 50, ..., 300 of 350
    check(inst, "dual", sparse, 350, dev=d)
