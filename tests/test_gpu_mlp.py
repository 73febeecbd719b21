"""GPU parity of the MLP policies (argmax and Gumbel-max) against the CPU oracle
through the C ABI.  The oracle scores in the reference FP32 order (one fmaf
chain per output from its bias); the kernels score faster and re-score near
ties in that order, so actions, pass counts, final stock and total cost must be
identical."""
import numpy as np
import pytest
import torch

import oracle
import paper_2406_01939_b300 as pic
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.session import DeviceInstance
from paper_2406_01939_b300.synth import Policy

pytestmark = pytest.mark.gpu


def small(seed, T, N, K, R, fill=0.9):
    inst = synth.make_instance(T, N, K, R, seed=seed, stock="poisson", fill=fill)
    return inst, synth.make_mlp(N, R, seed=seed)


def policies(mlp, seed):
    return [Policy("mlp", mlp=mlp), Policy("gumbel", mlp=mlp, seed=1000 + seed, traj=seed % 3)]


@pytest.mark.parametrize("N", [8, 33, 64, 100])
def test_sequential_mlp_bit_exact(N):
    inst, mlp = small(N, 1500, N, 30, 11)
    d = DeviceInstance(inst)
    for pol in policies(mlp, N):
        want = oracle.seq_sim(inst, pol)
        got = d.simulate(pol, "sequential")
        np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["actions"])
        np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), want["x_final"])
        assert got["total_cost"] == want["total_cost"] and got["lost"] == want["lost"]


@pytest.mark.parametrize("N", [8, 64])
def test_picard_mlp_iterates_and_fixed_point(N):
    """Pass count, fixed point and every intermediate cache alpha^k equal the
    oracle's (Algorithm 1 with the same blocks)."""
    inst, mlp = small(7 * N, 1200, N, 20, 9)
    d = DeviceInstance(inst)
    for pol in policies(mlp, N):
        M = 40
        want = oracle.picard_chunked(inst, pol, M, record=True)
        seq = oracle.seq_sim(inst, pol)
        got = d.simulate(pol, "picard", num_chunks=M)
        np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
        assert got["iters"] == want["iters"]
        assert got["total_cost"] == seq["total_cost"]
        np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])
        for k in (1, 2, want["iters"] // 2):
            g = d.simulate(pol, "picard", num_chunks=M, max_iters=k, raise_on_error=False)
            np.testing.assert_array_equal(g["actions"].cpu().numpy(), want["iterates"][k - 1])


def test_picard_mlp_windows_and_chunk_counts():
    inst, mlp = small(3, 2000, 32, 15, 6)
    d = DeviceInstance(inst)
    pol = Policy("mlp", mlp=mlp)
    seq = oracle.seq_sim(inst, pol)["actions"]
    for M in (1, 13, 2000):
        want = oracle.picard_chunked(inst, pol, M)
        for W in (1, 5, 64):
            got = d.simulate(pol, "picard", num_chunks=M, seg_window=W)
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq)
            assert got["iters"] == want["iters"]


def test_mlp_full_size_whole_trajectory_against_oracle():
    """T=2^18, N=64, K=2,000, R=500 MLP workload, the whole trajectory against
    the oracle's sequential simulation (every action, final stock, cost, lost
    count): Picard in the benchmark's configuration (4,096 chunks, max_steps
    window of 16,384 orders, segment window 4) and with 1,024 chunks, and the GPU
    sequential simulator with one warp and with four warps per decision."""
    inst, mlp = synth.mlp_medium(0)
    d = DeviceInstance(inst)
    pol = Policy("mlp", mlp=mlp)
    want = oracle.seq_sim(inst, pol)
    runs = [d.simulate(pol, "picard", num_chunks=4096, max_steps=16384, seg_window=4),
            d.simulate(pol, "picard", num_chunks=1024),
            d.simulate(pol, "sequential"),
            d.simulate(pol, "sequential", flags=pic.PIC_FLAG_WARP_GROUP)]
    for got in runs:
        np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["actions"])
        np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), want["x_final"])
        assert got["total_cost"] == want["total_cost"] and got["lost"] == want["lost"]


@pytest.mark.parametrize("N", [24, 32, 64])
def test_tensor_core_tiles_bit_exact(N):
    """PIC_FLAG_TC: long runs with ample stock are scored 16 orders at a time on
    the tensor cores; the actions, pass counts and iterates are the oracle's
    (rows whose top-2 margin is within the error bound are re-scored in FP32).
    The saturated-state table is turned off (PIC_FLAG_NO_SAT): with every
    warehouse stocked it would take these decisions instead of the tiles."""
    inst = synth.make_instance(12000, N, 6, 17, seed=N, stock="poisson", fill=1.2)
    mlp = synth.make_mlp(N, 17, seed=N)
    d = DeviceInstance(inst)
    for pol in policies(mlp, N):
        seq = oracle.seq_sim(inst, pol)
        rec = oracle.picard_chunked(inst, pol, 12, record=True)
        for M in (3, 12):
            want = rec if M == 12 else oracle.picard_chunked(inst, pol, M)
            got = d.simulate(pol, "picard", num_chunks=M, flags=pic.PIC_FLAG_TC | pic.PIC_FLAG_NO_SAT)
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
            np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])
            assert got["iters"] == want["iters"] and got["total_cost"] == seq["total_cost"]
            assert got["tc_decisions"] > 0  # the tiles were used
            assert got["tc_decisions"] + got["rescored"] <= got["mlp_calls"]
        for k in (1, 2):
            g = d.simulate(pol, "picard", num_chunks=12, max_iters=k, flags=pic.PIC_FLAG_TC | pic.PIC_FLAG_NO_SAT,
                           raise_on_error=False)
            np.testing.assert_array_equal(g["actions"].cpu().numpy(), rec["iterates"][k - 1])


def test_tensor_core_tiles_with_low_stock_and_ties():
    """Scarce stock (features change with every decrement, tiles stop early or
    are not started) and a scorer with exact ties (W2 = 0: every stocked
    warehouse scores b2; ties go to the lowest index, which the tiles must leave
    to the FP32 scorer)."""
    N = 16
    inst = synth.make_instance(6000, N, 4, 9, seed=5, stock="poisson", fill=0.3)
    mlp = synth.make_mlp(N, 9, seed=5)
    d = DeviceInstance(inst)
    pol = Policy("mlp", mlp=mlp)
    seq = oracle.seq_sim(inst, pol)
    got = d.simulate(pol, "picard", num_chunks=4, flags=pic.PIC_FLAG_TC | pic.PIC_FLAG_NO_SAT)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
    flat = synth.MLPParams(mlp.W1, mlp.b1, np.zeros_like(mlp.W2), np.zeros_like(mlp.b2), mlp.E)
    inst2 = synth.make_instance(6000, N, 4, 9, seed=6, stock="poisson", fill=2.0)
    d2 = DeviceInstance(inst2)
    pol2 = Policy("mlp", mlp=flat)
    seq2 = oracle.seq_sim(inst2, pol2)
    got2 = d2.simulate(pol2, "picard", num_chunks=4, flags=pic.PIC_FLAG_TC | pic.PIC_FLAG_NO_SAT)
    np.testing.assert_array_equal(got2["actions"].cpu().numpy(), seq2["actions"])
    assert got2["tc_decisions"] == 0 or got2["rescored"] > 0


@pytest.mark.parametrize("N", [8, 33, 64, 100])
def test_saturated_state_table_exact(N):
    """Products holding at least 32 units at every warehouse take their scores
    from the per-region table (built by the scorer itself); other products run
    the scorer.  Sequential and Picard paths equal the oracle with and without
    the table (PIC_FLAG_NO_SAT), and the table is used only by default."""
    inst, mlp = small(3 * N, 3000, N, 12, 9, fill=0.9)
    x0 = inst.x0.copy()
    x0[: inst.K // 2] += 60  # the popular half saturated for a while, the rest not
    inst.x0 = x0
    d = DeviceInstance(inst)
    for pol in policies(mlp, N):
        want = oracle.seq_sim(inst, pol)
        M = 25
        iters = oracle.picard_chunked(inst, pol, M)["iters"]
        for flags in (0, pic.PIC_FLAG_NO_SAT):
            for mode in ("sequential", "picard"):
                got = d.simulate(pol, mode, num_chunks=M, flags=flags)
                np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["actions"])
                np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), want["x_final"])
                assert got["total_cost"] == want["total_cost"]
                if mode == "picard":
                    assert got["iters"] == iters
                if flags:
                    assert got["sat_decisions"] == 0
                else:
                    assert 0 < got["sat_decisions"] < got["policy_calls"]


@pytest.mark.parametrize("N", [8, 33, 64, 100])
def test_four_warp_decisions_bit_exact(N):
    """PIC_FLAG_WARP_GROUP: four warps share each decision (same operations in
    the same order).  Sequential and Picard paths, with and without the window
    and the saturated-state table, equal the oracle; N > 64 falls back to one
    warp per decision."""
    inst, mlp = small(5 * N, 3000, N, 14, 9, fill=0.9)
    x0 = inst.x0.copy()
    x0[:3] += 40  # a few products saturated for a while (table decisions)
    inst.x0 = x0
    d = DeviceInstance(inst)
    G = pic.PIC_FLAG_WARP_GROUP
    for pol in policies(mlp, N):
        want = oracle.seq_sim(inst, pol)
        got = d.simulate(pol, "sequential", flags=G)
        np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["actions"])
        np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), want["x_final"])
        rec = oracle.picard_chunked(inst, pol, 30, record=True)
        for M, ms in ((30, 0), (100, 0), (100, 300)):
            # the oracle's pass count for this chunking (independent of the flags)
            ref = rec if (M, ms) == (30, 0) else (oracle.picard_windowed(inst, pol, M, ms) if ms else
                                                  oracle.picard_chunked(inst, pol, M))
            for flags in (G, G | pic.PIC_FLAG_NO_SAT):
                got = d.simulate(pol, "picard", num_chunks=M, max_steps=ms, flags=flags)
                np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["actions"])
                np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), want["x_final"])
                assert got["iters"] == ref["iters"] and got["total_cost"] == want["total_cost"]
        for k in (1, 3):
            g = d.simulate(pol, "picard", num_chunks=30, max_iters=k, flags=G, raise_on_error=False)
            np.testing.assert_array_equal(g["actions"].cpu().numpy(), rec["iterates"][k - 1])


def _bf(v):
    return synth.f32_to_bf16(np.asarray(v, np.float32))


def adversarial_mlp(N, R):
    """Weights on which the fast layer-2 order and the reference order rank two
    warehouses differently.  h_j = 1 for every hidden unit (W1 = 0, b1 = 1).
    Warehouse 0: b2 = 2^24 and W2[:, 0] = 1; the reference chain from b2 rounds
    every step back to 2^24 (ties to even), while any order that sums the 256
    ones first gives 2^24 + 256.  Warehouse 1: W2[0, 1] = 2^24, W2[1, 1] = 128,
    2^24 + 128 in every order.  The other warehouses score 0.  So the reference
    sends an order to warehouse 1 while it has stock, and the fast scores alone
    would send it to warehouse 0."""
    H = 256
    W1 = np.zeros((2 * N + 16, H))
    W2 = np.zeros((H, N))
    b2 = np.zeros(N)
    W2[:, 0] = 1.0
    b2[0] = 2.0 ** 24
    W2[0, 1] = 2.0 ** 24
    W2[1, 1] = 128.0
    return synth.MLPParams(_bf(W1), _bf(np.ones(H)), _bf(W2), _bf(b2), _bf(np.zeros((R, 16))), H)


@pytest.mark.parametrize("N", [8, 64, 100])
def test_near_ties_take_the_reference_order(N):
    """On adversarial_mlp the fast order disagrees with the reference on every
    decision where warehouses 0 and 1 both hold stock: the bound flags each one
    as a near tie and the re-score gives the oracle's action.  Every decision
    path: sequential, Picard, four warps per decision, tensor-core tiles, with
    and without the saturated-state table (whose scores are exact), argmax and
    Gumbel-max."""
    inst = synth.make_instance(3000, N, 4, 3, seed=N, stock="poisson", fill=0.6)
    mlp = adversarial_mlp(N, 3)
    d = DeviceInstance(inst)
    G, TC, NS = pic.PIC_FLAG_WARP_GROUP, pic.PIC_FLAG_TC, pic.PIC_FLAG_NO_SAT
    for pol in policies(mlp, N):
        want = oracle.seq_sim(inst, pol)
        a = want["actions"]
        # the reference picks warehouse 1 while it is stocked, then warehouse 0
        assert (a == 1).sum() > 10 and (a == 0).sum() > 0
        iters = oracle.picard_chunked(inst, pol, 30)["iters"]
        runs = [("sequential", 0), ("sequential", NS), ("picard", 0), ("picard", NS)]
        if N <= 64:
            runs += [("sequential", G | NS), ("picard", G | NS), ("picard", TC | NS)]
        for mode, flags in runs:
            got = d.simulate(pol, mode, num_chunks=30, flags=flags)
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), a, err_msg=f"{mode} {flags}")
            np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), want["x_final"])
            assert got["total_cost"] == want["total_cost"]
            if mode == "picard":
                assert got["iters"] == iters
            if flags & NS:
                assert got["near_ties"] > 0, (mode, flags)
