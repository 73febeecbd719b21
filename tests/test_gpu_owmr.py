"""GPU parity of the OWMR simulator (Appendix B) against the CPU oracle, through
the C ABI.  Actions (2 q + r), final state, replenishments, lost and shipped
units are compared bit for bit; the Picard pass count and the number of network
calls must equal the oracle walk's (both memoise per step with the same rule)."""
import numpy as np
import pytest
import torch

import paper_2406_01939_b300 as pic
from oracle import owmr as ow
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.owmr import DeviceOwmr, DeviceOwmrNet

pytestmark = pytest.mark.gpu


def rand_inst(seed, T, N, theorem=True, a=0.0):
    rng = np.random.default_rng(seed)
    cap = rng.integers(1, 12, N)
    Sl = np.minimum(cap, rng.integers(1, 12, N))
    sl = np.array([rng.integers(0, v + 1) for v in Sl])
    s = int(cap.max() + rng.integers(0, 6)) if theorem else int(rng.integers(0, 4))
    S = s + int(rng.integers(1, 4 * N + 40))
    return synth.make_owmr(T, N, seed=seed, a=a, demand="small", s_loc=sl, S_loc=Sl, cap=cap,
                           s=s, S=S, X0=int(rng.integers(s + 1, S + 1)),
                           x0r=np.array([rng.integers(0, c + 1) for c in cap]))


def procs_of(N, P):
    return (np.arange(N) % P).astype(np.int32)


def check(inst, net, P, dev=None, dnet=None, **kw):
    seq = ow.seq_sim(inst, net)
    want = ow.picard_walk(inst, net, procs_of(inst.N, P))
    d = dev or DeviceOwmr(inst)
    got = d.simulate(dnet if dnet is not None else net, num_procs=P, **kw)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
    np.testing.assert_array_equal(got["state"].cpu().numpy(), seq["x_final"])
    assert (got["R"], got["lost"], got["shipped"]) == (seq["R"], seq["lost"], seq["shipped"])
    assert got["iters"] == want["iters"], (got["iters"], want["iters"])
    if net is not None:
        assert got["policy_calls"] == want["evals"], (got["policy_calls"], want["evals"])
    return got, want


@pytest.mark.parametrize("N", [1, 5, 33, 100])
def test_no_network_random_bit_exact(N):
    for trial in range(4):
        T = [0, 1, 777, 5000][trial]
        inst = rand_inst(1000 * N + trial, T, N, theorem=bool(trial % 2))
        d = DeviceOwmr(inst)
        for P in sorted({N, max(1, N // 2), 1, min(N, 3)}):
            if -(-N // P) > 128:
                continue
            check(inst, None, P, dev=d)


def test_network_bit_exact_and_calls():
    """H = 64 and 512, ragged groups (N = 45 processors over several lanes),
    skewed store weights; the same calls as the oracle's memo."""
    for H, T, N, a in ((64, 3000, 45, 0.0), (512, 1500, 37, 0.02), (128, 2500, 70, 0.0),
                       (256, 4000, 300, 0.0), (64, 30000, 2000, 0.0)):
        inst = rand_inst(H + N, T, N, theorem=H != 128, a=a)
        net = synth.make_owmr_net(H, seed=H)
        d = DeviceOwmr(inst)
        dn = DeviceOwmrNet(net)
        for P in (N, max(1, N // 3)):
            check(inst, net, P, dev=d, dnet=dn)


def test_every_iterate_matches_algorithm_1():
    inst = rand_inst(7, 1200, 9, theorem=False)
    net = synth.make_owmr_net(64, seed=2)
    d = DeviceOwmr(inst)
    for nn in (None, net):
        want = ow.picard_literal(inst, nn, procs_of(9, 9), record=True)
        for k in range(1, want["iters"] + 1):
            got = d.simulate(nn, num_procs=9, max_iters=k, raise_on_error=False)
            assert got["status"] == (pic.PIC_OK if k == want["iters"] else pic.PIC_ERR_NOT_CONVERGED)
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["iterates"][k - 1])


def test_sequential_mode_bit_exact():
    for seed, N, H in ((1, 8, 0), (2, 50, 64), (3, 20, 512)):
        inst = rand_inst(seed, 2000, N, theorem=seed != 2)
        net = synth.make_owmr_net(H, seed=seed) if H else None
        seq = ow.seq_sim(inst, net)
        got = DeviceOwmr(inst).simulate(net, mode="sequential")
        np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
        np.testing.assert_array_equal(got["state"].cpu().numpy(), seq["x_final"])
        assert (got["R"], got["lost"], got["shipped"]) == (seq["R"], seq["lost"], seq["shipped"])


def test_warm_start():
    inst = rand_inst(9, 4000, 30)
    net = synth.make_owmr_net(64, seed=9)
    seq = ow.seq_sim(inst, net)["actions"]
    d = DeviceOwmr(inst)
    assert d.simulate(net, alpha_init=seq)["iters"] == 1
    rng = np.random.default_rng(0)
    init = (2 * rng.integers(0, 5, inst.T) + rng.integers(0, 2, inst.T)).astype(np.int32)
    want = ow.picard_walk(inst, net, procs_of(30, 30), alpha_init=init)
    got = d.simulate(net, alpha_init=init)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq)
    assert got["iters"] == want["iters"] and got["policy_calls"] == want["evals"]


def test_window_bit_exact_and_passes():
    """The max_steps window: same iterates, passes and network calls as the
    oracle's windowed walk, for windows from one step to the horizon."""
    net = synth.make_owmr_net(64, seed=12)
    for seed, T, N in ((21, 3000, 24), (22, 5000, 70), (23, 777, 5)):
        inst = rand_inst(seed, T, N, theorem=seed != 22)
        d = DeviceOwmr(inst)
        dn = DeviceOwmrNet(net)
        for W in (1, 37, 500, T):
            for nn, dd in ((None, None), (net, dn)):
                seq = ow.seq_sim(inst, nn)
                want = ow.picard_walk(inst, nn, procs_of(N, N), window=W)
                got = d.simulate(dd, max_steps=W)
                np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
                np.testing.assert_array_equal(got["state"].cpu().numpy(), seq["x_final"])
                assert got["iters"] == want["iters"], (W, got["iters"], want["iters"])
                if nn is not None:
                    assert got["policy_calls"] == want["evals"]
    inst = rand_inst(24, 1500, 9, theorem=False)
    d = DeviceOwmr(inst)
    want = ow.picard_literal(inst, net, procs_of(9, 9), record=True, window=100)
    for k in range(1, want["iters"] + 1, 3):
        got = d.simulate(net, max_iters=k, max_steps=100, raise_on_error=False)
        np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["iterates"][k - 1])


def test_window_scaled_base_case():
    """The base case at a tenth of its size (365,000 steps, 400 stores) with a
    window of 16,000 steps: the oracle's passes and network calls (each step's
    network evaluated about once)."""
    inst, _ = synth.owmr_base(0, T=365_000, N=400, H=64)
    inst.S = inst.s + 7_000
    net = synth.make_owmr_net(64, seed=0)
    want = ow.picard_walk(inst, net, procs_of(400, 400), window=16_000)
    d = DeviceOwmr(inst)
    got = d.simulate(net, max_steps=16_000)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["actions"])
    assert got["iters"] == want["iters"] and got["policy_calls"] == want["evals"]


def test_many_groups_per_cta():
    """More processors than 32 per SM: each CTA walks several groups."""
    inst = rand_inst(11, 30000, 6000)
    check(inst, None, 6000)


def test_invalid_inputs():
    inst = rand_inst(5, 100, 4)
    bad = rand_inst(5, 100, 4)
    bad.ret = bad.ret.copy()
    bad.ret[7] = 4
    with pytest.raises(pic.PicError) as e:
        DeviceOwmr(bad)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG and "ret" in str(e.value)
    bad = rand_inst(5, 100, 4)
    bad.Sl = bad.cap + 1
    with pytest.raises(pic.PicError) as e:
        DeviceOwmr(bad)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG
    d = DeviceOwmr(inst)
    net = synth.make_owmr_net(64, seed=0)
    net.H = 96
    with pytest.raises(pic.PicError) as e:
        d.simulate(net)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG
    with pytest.raises(pic.PicError) as e:
        d.simulate(None, alpha_init=np.full(inst.T, -2, np.int32))
    assert e.value.status == pic.PIC_ERR_INVALID_ARG
    big = rand_inst(6, 100, 200)
    with pytest.raises(pic.PicError) as e:
        DeviceOwmr(big).simulate(None, num_procs=1)
    assert e.value.status == pic.PIC_ERR_UNSUPPORTED


def test_base_case_full_size():
    """Appendix B.3's base case (T = 3,650,000, 4,000 stores, one processor
    each): without the network against the oracle's sequential path and pass
    count (Theorem B.1: 2R + 2 passes here); with the width-512 network, the
    Picard path equals the GPU sequential path over the whole horizon and the
    oracle's sequential path on the first 20,000 steps (a prefix of the path
    depends only on the prefix of the disturbances)."""
    inst, net = synth.owmr_base(0)
    seq = ow.seq_sim(inst)
    d = DeviceOwmr(inst)
    got = d.simulate(None)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
    np.testing.assert_array_equal(got["state"].cpu().numpy(), seq["x_final"])
    assert got["iters"] <= 2 * seq["R"] + 2
    dn = DeviceOwmrNet(net)
    pg = d.simulate(dn, max_steps=80_000)
    sg = d.simulate(dn, mode="sequential")
    assert torch.equal(pg["actions"], sg["actions"]) and torch.equal(pg["state"], sg["state"])
    assert pg["R"] == sg["R"] and pg["lost"] == sg["lost"]
    Tp = 20_000
    pre = synth.OwmrInstance(Tp, inst.N, inst.ret[:Tp], inst.dem[:Tp], inst.ex[:Tp], inst.cap,
                             inst.x0r, inst.sl, inst.Sl, inst.X0, inst.s, inst.S)
    np.testing.assert_array_equal(pg["actions"][:Tp].cpu().numpy(), ow.seq_sim(pre, net)["actions"])


def test_output_layer_near_ties_take_the_reference_order():
    """A network whose fast output layer and reference chain disagree: h2_j = 1
    (W1 = 0, b1 = 0, W2 = 0, b2 = 1), w3_0 = -2^24, w3_1..3 = 1, other w3 = 0,
    b3 = 2^24.  The reference chain gives 2^24 - 2^24 + 1 + 1 + 1 = 3; the
    group of eight first gives -2^24 (each +1 rounds back), then z = 0.  Every
    q with room for it differs, so the kernels must detect the undecided floor
    and re-evaluate z in the reference order: actions equal the oracle's, in
    Picard and sequential mode."""
    H = 64
    bf = lambda v: synth.f32_to_bf16(np.asarray(v, np.float32))
    w3 = np.zeros(H)
    w3[0] = -(2.0 ** 24)
    w3[1:4] = 1.0
    net = synth.OwmrNet(H, bf(np.zeros((3, H))), bf(np.zeros(H)), bf(np.zeros((H, H))),
                        bf(np.ones(H)), bf(w3), bf([2.0 ** 24]))
    assert ow.mlp(net, 1, 1, 1) == 3.0
    inst = rand_inst(77, 3000, 12, theorem=False)
    seq = ow.seq_sim(inst, net)
    base_only = ow.seq_sim(inst, None)
    assert (seq["actions"] != base_only["actions"]).any()  # the network moves q
    d = DeviceOwmr(inst)
    for mode in ("picard", "sequential"):
        got = d.simulate(net, mode=mode)
        np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
        np.testing.assert_array_equal(got["state"].cpu().numpy(), seq["x_final"])
        assert got["near_ties"] > 0
