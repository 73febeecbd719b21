"""Pins for the oracle's max_steps window (Appendix A.3) on contiguous blocks.
CPU only."""
import itertools

import numpy as np

import oracle
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.synth import Instance, Policy


def rand_inst(rng, T, N, K, R):
    return Instance(T, N, K, R, rng.integers(0, K, T).astype(np.int32),
                    rng.integers(0, R, T).astype(np.int32),
                    rng.integers(0, 5, (K, N)).astype(np.int32),
                    rng.integers(1, 6, (R, N)).astype(np.int32),
                    rng.integers(0, 4, (K, N)).astype(np.int32))


def all_policies(inst, seed):
    mlp = synth.make_mlp(inst.N, inst.R, seed=seed)
    return [Policy("greedy"), Policy("dual"), Policy("mlp", mlp=mlp),
            Policy("gumbel", mlp=mlp, seed=seed, traj=2)]


def test_window_covering_the_horizon_is_algorithm_1():
    """max_steps >= T: every pass evaluates every block, so the iterates and the
    pass count are those of Algorithm 1."""
    rng = np.random.default_rng(21)
    for trial in range(30):
        inst = rand_inst(rng, int(rng.integers(1, 60)), int(rng.integers(1, 5)), 3, 3)
        for pol in all_policies(inst, trial):
            M = int(rng.integers(1, inst.T + 1))
            a = oracle.picard_windowed(inst, pol, M, max_steps=inst.T + int(rng.integers(0, 5)),
                                       record=True)
            b = oracle.picard_chunked(inst, pol, M, record=True)
            assert a["iters"] == b["iters"]
            np.testing.assert_array_equal(a["iterates"], b["iterates"])


def test_window_fixed_point_is_sequential_path():
    """Whatever the window, the loop returns the sequential path (the window
    only moves past blocks that reached their fixed point from an exact
    prefix)."""
    rng = np.random.default_rng(22)
    for trial in range(40):
        inst = rand_inst(rng, int(rng.integers(1, 80)), int(rng.integers(1, 6)), 4, 3)
        for pol in all_policies(inst, trial):
            seq = oracle.seq_sim(inst, pol)["actions"]
            M = int(rng.integers(1, inst.T + 1))
            for ms in (1, int(rng.integers(1, inst.T + 1)), inst.T):
                out = oracle.picard_windowed(inst, pol, M, max_steps=ms)
                assert out["converged"]
                np.testing.assert_array_equal(out["actions"], seq)


def test_one_block_per_window_takes_at_most_two_passes_per_block():
    """max_steps <= L: each window holds one block, whose prefix is exact when
    the window reaches it; one pass computes it and at most one more confirms
    it, so at most 2 M passes, and the first pass of each window already holds
    the sequential actions of that block."""
    rng = np.random.default_rng(23)
    for trial in range(30):
        inst = rand_inst(rng, int(rng.integers(4, 80)), int(rng.integers(1, 5)), 3, 4)
        M = int(rng.integers(1, inst.T + 1))
        L = -(-inst.T // M)
        for pol in all_policies(inst, trial):
            seq = oracle.seq_sim(inst, pol)["actions"]
            out = oracle.picard_windowed(inst, pol, M, max_steps=int(rng.integers(1, L + 1)),
                                         record=True)
            nb = -(-inst.T // L)
            assert out["iters"] <= 2 * nb
            np.testing.assert_array_equal(out["actions"], seq)
            np.testing.assert_array_equal(out["iterates"][0][:L], seq[:L])


def test_window_exhaustive_tiny_family():
    """T = 5, N = 2, K = 2, x0 in {0,1,2}^4, every product sequence, every
    M and max_steps: the sequential path."""
    T, N, K = 5, 2, 2
    cost = np.array([[3, 1], [1, 3]], np.int32)
    reg = np.array([0, 1, 0, 0, 1], np.int32)
    lam = np.array([[0, 2], [1, 0]], np.int32)
    n = 0
    for x0f in itertools.product(range(3), repeat=K * N):
        for prodv in itertools.product(range(K), repeat=T):
            inst = Instance(T, N, K, 2, np.array(prodv, np.int32), reg,
                            np.array(x0f, np.int32).reshape(K, N), cost, lam)
            for kind in ("greedy", "dual"):
                pol = Policy(kind)
                seq = oracle.seq_sim(inst, pol)["actions"]
                for M in range(1, T + 1):
                    for ms in range(1, T + 1):
                        np.testing.assert_array_equal(
                            oracle.picard_windowed(inst, pol, M, ms)["actions"], seq)
            n += 1
    assert n == 81 * 32


def test_window_pass_count_closed_form_with_state_free_policy():
    """Greedy with ample stock never depends on the state, so a block is final
    after its first evaluation and every order is fulfilled (so the first order
    of a newly evaluated block changes).  The window then covers
    B = ceil(max_steps / L) blocks from a block boundary; each window takes one
    pass that changes its new blocks and one that confirms them:
    2 ceil(nblocks / B) passes, with the window starting at 0 and moving by B
    blocks."""
    rng = np.random.default_rng(24)
    for trial in range(60):
        T = int(rng.integers(1, 120))
        N, K = int(rng.integers(1, 5)), 3
        inst = rand_inst(rng, T, N, K, 3)
        inst.x0 = np.full((K, N), T, np.int32)
        M = int(rng.integers(1, T + 1))
        L = -(-T // M)
        nb = -(-T // L)
        ms = int(rng.integers(1, T + 1))
        B = -(-ms // L)
        out = oracle.picard_windowed(inst, Policy("greedy"), M, ms, record=True)
        assert out["iters"] == 2 * (-(-nb // B)), (T, M, ms, out["iters"])
        for p in range(out["iters"]):
            w = p // 2  # window index of pass p (0-based)
            done = min(T, (w + 1) * B * L)
            np.testing.assert_array_equal(out["iterates"][p][:done] >= 0, True)
            np.testing.assert_array_equal(out["iterates"][p][done:], -1)
