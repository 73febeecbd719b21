"""PIC_FLAG_WAVE: MLP decisions in CTA-wide waves on the tensor cores (tcgen05),
each kept only when its top-2 margin exceeds twice the bound on the difference
from the reference FP32 order, else re-scored by the FP32 scorer.  Actions,
pass counts, every intermediate cache, final stock and costs must equal the
oracle's (Algorithm 1 on the same chunks; the sequential simulation)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2406_01939_b300 as pic
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.session import DeviceBatch, DeviceInstance
from paper_2406_01939_b300.synth import Policy

pytestmark = pytest.mark.gpu

W = pic.PIC_FLAG_WAVE | pic.PIC_FLAG_TC  # every wave on the tensor cores


def policies(mlp, seed):
    return [Policy("mlp", mlp=mlp), Policy("gumbel", mlp=mlp, seed=500 + seed, traj=seed % 4)]


@pytest.mark.parametrize("N", [8, 32, 48, 64])
def test_wave_picard_matches_oracle(N):
    inst = synth.make_instance(3000, N, 25, 11, seed=N, stock="poisson", fill=0.9)
    x0 = inst.x0.copy()
    x0[:4] += 45  # a few products saturated for a while (table decisions in the waves)
    inst.x0 = x0
    mlp = synth.make_mlp(N, 11, seed=N)
    d = DeviceInstance(inst)
    for pol in policies(mlp, N):
        seq = oracle.seq_sim(inst, pol)
        for M, flags in ((30, W), (30, W | pic.PIC_FLAG_NO_SAT), (200, W), (3000, W),
                         (200, pic.PIC_FLAG_WAVE), (200, pic.PIC_FLAG_WAVE | pic.PIC_FLAG_NO_TC)):
            want = oracle.picard_chunked(inst, pol, M)
            got = d.simulate(pol, "picard", num_chunks=M, flags=flags)
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
            np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])
            assert got["total_cost"] == seq["total_cost"] and got["lost"] == seq["lost"]
            assert got["iters"] == want["iters"], (M, flags, got["iters"], want["iters"])
            assert got["wave"]  # the result names the kernel that ran
            if flags & pic.PIC_FLAG_TC:
                assert got["tc_decisions"] > 0
            if flags & pic.PIC_FLAG_NO_TC:
                assert got["tc_decisions"] == 0
            assert got["tc_decisions"] + got["sat_decisions"] + got["rescored"] <= got["policy_calls"]


def test_wave_every_iterate_and_windows():
    """Every intermediate cache alpha^k equals Algorithm 1's, and the max_steps
    window gives the oracle's pass count."""
    N = 32
    inst = synth.make_instance(2500, N, 20, 9, seed=3, stock="poisson", fill=0.8)
    mlp = synth.make_mlp(N, 9, seed=3)
    d = DeviceInstance(inst)
    for pol in policies(mlp, 3):
        rec = oracle.picard_chunked(inst, pol, 40, record=True)
        for k in (1, 2, 3, rec["iters"] // 2):
            g = d.simulate(pol, "picard", num_chunks=40, max_iters=k, flags=W, raise_on_error=False)
            np.testing.assert_array_equal(g["actions"].cpu().numpy(), rec["iterates"][k - 1])
        for ms in (300, 1000):
            want = oracle.picard_windowed(inst, pol, 100, ms)
            got = d.simulate(pol, "picard", num_chunks=100, max_steps=ms, flags=W)
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["actions"])
            assert got["iters"] == want["iters"]


def test_wave_near_ties_take_the_reference_order():
    """The adversarial weights on which a 256-term sum in another order ranks
    warehouses 0 and 1 the other way: every such wave row is a near tie, and the
    FP32 scorer's reference order gives the oracle's action."""
    from test_gpu_mlp import adversarial_mlp
    N = 16
    inst = synth.make_instance(2000, N, 4, 3, seed=9, stock="poisson", fill=0.6)
    mlp = adversarial_mlp(N, 3)
    d = DeviceInstance(inst)
    for pol in policies(mlp, 1):
        seq = oracle.seq_sim(inst, pol)
        got = d.simulate(pol, "picard", num_chunks=20, flags=W | pic.PIC_FLAG_NO_SAT)
        np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
        assert got["rescored"] > 0


def test_wave_batch_mixed_policies():
    """A batch of greedy, bid-price, MLP and Gumbel trajectories in one wave
    launch: each trajectory equals the oracle's sequential simulation, with the
    pass count pic_simulate gives it alone."""
    N, K, R = 32, 10, 7
    rng = np.random.default_rng(5)
    mlp = synth.make_mlp(N, R, seed=5)
    insts, pols = [], []
    for b, kind in enumerate(["greedy", "mlp", "dual", "gumbel", "mlp", "greedy", "gumbel"]):
        T = int(rng.integers(500, 4000))
        insts.append(synth.make_instance(T, N, K, R, seed=100 + b, stock="poisson", with_lam=True))
        pols.append(Policy(kind, mlp=mlp if kind in ("mlp", "gumbel") else None, seed=7 + b, traj=b))
    db = DeviceBatch(insts)
    wants = [oracle.seq_sim(inst, pol) for inst, pol in zip(insts, pols)]
    iters = [oracle.picard_chunked(inst, pol, min(24, inst.T))["iters"] for inst, pol in zip(insts, pols)]
    for flags in (W, W | pic.PIC_FLAG_NO_SAT):
        got = db.simulate(pols, "picard", num_chunks=24, flags=flags)
        assert got["wave"]
        acts = db.split(got["actions"].cpu().numpy())
        xf = db.split_stock(got["final_stock"].cpu().numpy())
        for b, want in enumerate(wants):
            np.testing.assert_array_equal(acts[b], want["actions"], err_msg=f"trajectory {b}")
            np.testing.assert_array_equal(xf[b], want["x_final"])
            assert got["traj"][b]["total_cost"] == want["total_cost"]
            assert got["traj"][b]["iters"] == iters[b], b


def test_wave_batch_uneven_full_size_equals_default_kernel():
    """The 512-trajectory uneven batch (T_b ~ U{16,384..262,144}, N = 32, half
    greedy, half MLP): the wave launch gives the per-warp launch's paths, costs
    and pass counts, and its first MLP trajectory equals the oracle's."""
    insts, pols = synth.batch_uneven(0)
    db = DeviceBatch(insts)
    base = db.simulate(pols, "picard", num_chunks=64, flags=pic.PIC_FLAG_NO_WAVE)
    assert not base["wave"]
    for flags in (W, pic.PIC_FLAG_WAVE):
        got = db.simulate(pols, "picard", num_chunks=64, flags=flags)
        assert torch.equal(got["actions"], base["actions"])
        assert torch.equal(got["final_stock"], base["final_stock"])
        for b in range(len(insts)):
            assert got["traj"][b] == base["traj"][b], b
    want = oracle.seq_sim(insts[1], pols[1])
    np.testing.assert_array_equal(db.split(got["actions"].cpu().numpy())[1], want["actions"])
