"""GPU parity of Picard with the max_steps window (Appendix A.3) against the
oracle's windowed Algorithm 1: actions, every intermediate cache and the pass
count, for the integer and MLP policies."""
import numpy as np
import pytest
import torch

import oracle
import paper_2406_01939_b300 as pic
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.session import DeviceBatch, DeviceInstance
from paper_2406_01939_b300.synth import Instance, Policy

pytestmark = pytest.mark.gpu


def rand_inst(rng, T, N, K, R):
    return Instance(T, N, K, R, rng.integers(0, K, T).astype(np.int32),
                    rng.integers(0, R, T).astype(np.int32),
                    rng.integers(0, 7, (K, N)).astype(np.int32),
                    rng.integers(1, 10, (R, N)).astype(np.int32),
                    rng.integers(0, 4, (K, N)).astype(np.int32))


def check(d, inst, pol, M, ms, cache=None, **kw):
    """cache: a dict living no longer than inst, holding the oracle's results
    for repeated checks of the same instance and policy."""
    cache = {} if cache is None else cache
    pk = (id(inst), pol.kind, pol.seed, pol.traj, id(pol.mlp))
    if pk + (M, ms) not in cache:
        cache[pk + (M, ms)] = oracle.picard_windowed(inst, pol, M, ms)
    if pk not in cache:
        cache[pk] = oracle.seq_sim(inst, pol)
    want, seq = cache[pk + (M, ms)], cache[pk]
    got = d.simulate(pol, "picard", num_chunks=M, max_steps=ms, **kw)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
    assert got["iters"] == want["iters"], (M, ms, got["iters"], want["iters"])
    assert got["total_cost"] == seq["total_cost"] and got["lost"] == seq["lost"]
    np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])
    return got, want


@pytest.mark.parametrize("N", [5, 33, 64, 100])
def test_window_integer_policies(N):
    rng = np.random.default_rng(N)
    for T, K, R in ((1, 1, 1), (37, 4, 5), (1000, 40, 7), (5000, 17, 40)):
        inst = rand_inst(rng, T, N, K, R)
        d = DeviceInstance(inst)
        cache = {}
        for kind in ("greedy", "dual"):
            for M in sorted({1, 7, max(1, T // 16), T}):
                L = -(-T // M)
                for ms in sorted({1, L, 3 * L + 5, T}):
                    for W in (1, 64):
                        check(d, inst, Policy(kind), M, ms, cache=cache, seg_window=W)
        # t_reset off: same iterates (t_reset only skips replays that reproduce the cache)
        check(d, inst, Policy("dual"), max(1, T // 16), max(1, T // 5), flags=pic.PIC_FLAG_NO_RESET)


def test_window_every_iterate():
    inst = synth.greedy_small(4)
    pol = Policy("greedy")
    M, ms = 64, 400
    want = oracle.picard_windowed(inst, pol, M, ms, record=True)
    d = DeviceInstance(inst)
    for k in range(1, want["iters"] + 1):
        got = d.simulate(pol, "picard", num_chunks=M, max_steps=ms, max_iters=k,
                         raise_on_error=False)
        assert got["status"] == (pic.PIC_OK if k == want["iters"] else pic.PIC_ERR_NOT_CONVERGED)
        np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["iterates"][k - 1])


@pytest.mark.parametrize("N", [8, 64])
def test_window_mlp_policies(N):
    inst = synth.make_instance(2500, N, 12, 9, seed=N, stock="poisson", fill=0.9)
    mlp = synth.make_mlp(N, 9, seed=N)
    d = DeviceInstance(inst)
    cache = {}
    for pol in (Policy("mlp", mlp=mlp), Policy("gumbel", mlp=mlp, seed=5, traj=1)):
        for M, ms in ((50, 1), (50, 120), (100, 700), (25, 2500)):
            check(d, inst, pol, M, ms, cache=cache)
        want = oracle.picard_windowed(inst, pol, 50, 300, record=True)
        for k in (1, 2, 5):
            got = d.simulate(pol, "picard", num_chunks=50, max_steps=300, max_iters=k,
                             raise_on_error=False)
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["iterates"][k - 1])


def test_window_rejected_where_unsupported():
    inst = synth.greedy_small(1)
    d = DeviceInstance(inst)
    with pytest.raises(pic.PicError) as e:
        d.simulate(Policy("greedy"), "picard", num_chunks=8, max_steps=-1)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG
    db = DeviceBatch([inst, synth.greedy_small(2)])
    with pytest.raises(pic.PicError) as e:
        db.simulate([Policy("greedy"), Policy("greedy")], "picard", num_chunks=8, max_steps=100)
    assert e.value.status == pic.PIC_ERR_UNSUPPORTED
    inst.cap = np.full(inst.N, 1000, np.int32)
    with pytest.raises(pic.PicError) as e:
        DeviceInstance(inst).simulate(Policy("greedy"), "picard", num_chunks=64, max_steps=100)
    assert e.value.status == pic.PIC_ERR_UNSUPPORTED


def test_window_mlp_medium_shape():
    """The MLP workload's shape (T = 2^18, N = 64, K = 2,000) with a window of 32
    chunks: the sequential GPU path, with fewer policy calls than without it."""
    inst, mlp = synth.mlp_medium(0)
    d = DeviceInstance(inst)
    pol = Policy("mlp", mlp=mlp)
    full = d.simulate(pol, "picard", num_chunks=1024)
    win = d.simulate(pol, "picard", num_chunks=1024, max_steps=32 * 256)
    assert torch.equal(full["actions"], win["actions"])
    assert win["policy_calls"] < full["policy_calls"]
    seq = d.simulate(pol, "sequential")
    assert torch.equal(seq["actions"], win["actions"])
