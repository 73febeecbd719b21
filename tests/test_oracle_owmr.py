"""Pins for the OWMR oracle (Appendix B): hand-derived traces, closed forms of
the (s, S) central policy, conservation, the network against an FP64
evaluation within its rounding bound, Prop. 1 and Theorem B.1 for the literal
Picard iteration under the retailer partition, and the walk organisation
against the literal iteration pass by pass."""
import numpy as np
import pytest

from oracle import owmr as ow
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.synth import OwmrInstance, OwmrNet


def inst_of(ret, dem, cap, x0r, sl, Sl, X0, s, S):
    a = lambda v: np.asarray(v, np.int32)
    return OwmrInstance(len(ret), len(cap), a(ret), a(dem), synth.demand_gaps(a(ret)), a(cap),
                        a(x0r), a(sl), a(Sl), X0, s, S)


def test_hand_trace_theorem_setting():
    """Two stores, s = 5 >= c_n = 5.  Derivation, per step (store, demand):
    t0 (0,2): y=1<=1, q=4-1=3, 9-3=6>5 -> r=0, store0=1+3=4, x0=6   -> 6
    t1 (1,4): y=1<=2, q=5-1=4, 6-4=2<=5 -> r=1, store1=1+4=5, x0=12  -> 9
    t2 (0,6): lost 2, y=0, q=4, 12-4=8>5 -> r=0, store0=4, x0=8       -> 8
    t3 (1,0): y=5>2, q=0, 8>5 -> r=0, x0=8                           -> 0
    t4 (1,3): y=2<=2, q=min(3, 5-2)=3, 8-3=5<=5 -> r=1, store1=5, x0=12 -> 7
    t5 (0,1): y=3>1, q=0, r=0, store0=3                              -> 0"""
    inst = inst_of([0, 1, 0, 1, 1, 0], [2, 4, 6, 0, 3, 1], [5, 5], [3, 5], [1, 2], [4, 5], 9, 5, 12)
    out = ow.seq_sim(inst)
    assert out["actions"].tolist() == [6, 9, 8, 0, 7, 0]
    assert out["x_final"].tolist() == [12, 3, 5]
    assert (out["R"], out["lost"], out["shipped"]) == (2, 2, 14)


def test_hand_trace_short_central_warehouse():
    """s = 0 < c_n: the retailer receives min(q, x0).  One store, c=5, (2, 5):
    t0 (0): q=5, 2-5<=0 r=1, recv 2 -> 2, x0=10       -> 11
    t1 (1): y=1, q=4, 6>0 r=0, recv 4 -> 5, x0=6       -> 8
    t2 (5): y=0, q=5, 1>0 r=0, recv 5 -> 5, x0=1       -> 10
    t3 (2): y=3>2, q=0, r=0 -> 3, x0=1                 -> 0
    t4 (3): y=0, q=5, 1-5<=0 r=1, recv 1 -> 1, x0=10   -> 11"""
    inst = inst_of([0] * 5, [0, 1, 5, 2, 3], [5], [0], [2], [5], 2, 0, 10)
    out = ow.seq_sim(inst)
    assert out["actions"].tolist() == [11, 8, 10, 0, 11]
    assert out["x_final"].tolist() == [10, 1]
    assert (out["R"], out["lost"], out["shipped"]) == (2, 0, 12)


def random_inst(rng, T, N, theorem=True, demand="small"):
    cap = rng.integers(1, 9, N)
    Sl = np.minimum(cap, rng.integers(1, 9, N))
    sl = np.array([rng.integers(0, v + 1) for v in Sl])
    s = int(cap.max() + rng.integers(0, 6)) if theorem else int(rng.integers(0, 4))
    S = s + int(rng.integers(1, 40))
    X0 = int(rng.integers(s + 1, S + 1))
    x0r = np.array([rng.integers(0, c + 1) for c in cap])
    inst = synth.make_owmr(T, N, seed=int(rng.integers(1 << 30)), demand=demand, s_loc=sl,
                           S_loc=Sl, cap=cap, s=s, S=S, X0=X0, x0r=x0r)
    return inst


def central_closed_form_ok(inst, act):
    """(s, S): x0 before step t is max(0, B - sum of q since the last
    replenishment), B = S after a replenishment, X0 before the first; r_t = 1
    exactly when that level minus q_t is at most s."""
    q, r = act >> 1, act & 1
    B, since = inst.X0, 0
    for t in range(inst.T):
        x0 = max(0, B - since)
        if bool(r[t]) != (x0 - q[t] <= inst.s):
            return False
        if r[t]:
            B, since = inst.S, 0
        else:
            since += int(q[t])
    return True


@pytest.mark.parametrize("theorem", [True, False])
def test_seq_invariants(theorem):
    rng = np.random.default_rng(3 + theorem)
    net = synth.make_owmr_net(64, seed=5)
    for trial in range(20):
        inst = random_inst(rng, int(rng.integers(1, 400)), int(rng.integers(1, 9)), theorem)
        for nn in (None, net):
            out = ow.seq_sim(inst, nn)
            act = out["actions"]
            assert central_closed_form_ok(inst, act)
            assert out["R"] == int((act & 1).sum())
            # conservation over the retailers: stock change = shipped - sold
            sold = int(inst.dem.sum()) - out["lost"]
            assert int(out["x_final"][1:].sum() - inst.x0r.sum()) == out["shipped"] - sold
            assert (out["x_final"][1:] <= inst.cap).all() and (out["x_final"] >= 0).all()
            assert ((act >> 1) <= inst.cap[inst.ret]).all() and (act >= 0).all()
            if theorem:  # x0 > s >= q: every request is shipped in full
                assert out["shipped"] == int((act >> 1).sum())
            assert out["evals"] == (inst.T if nn is not None else 0)


def test_no_orders_no_replenishment():
    inst = synth.make_owmr(500, 4, seed=1, demand="small", s_loc=0, S_loc=0, cap=6, s=3, S=50,
                           x0r=6)
    out = ow.seq_sim(inst)
    assert (out["actions"] == 0).all() and out["R"] == 0 and out["x_final"][0] == 50
    # each store sells its 6 units, then loses everything else
    per = [int(inst.dem[inst.ret == n].sum()) for n in range(4)]
    assert out["lost"] == sum(max(0, d - 6) for d in per)


def bf(x):
    return synth.f32_to_bf16(np.asarray(x, np.float32))


def const_net(H, b3):
    z = bf(np.zeros(1))
    return OwmrNet(H, bf(np.zeros(3 * H)), bf(np.zeros(H)), bf(np.zeros(H * H)),
                   bf(np.zeros(H)), bf(np.zeros(H)), bf([b3]))


def test_network_constant_output_special_cases():
    """All weights zero: z = b3 exactly.  b3 = 0.5 gives floor(base + 0.5) =
    base, the network-free rule; b3 = -0.75 gives max(0, base - 1), which is the
    network-free rule with S_n - 1 when s_n < S_n."""
    rng = np.random.default_rng(11)
    inst = random_inst(rng, 300, 5)
    plain = ow.seq_sim(inst)
    assert ow.mlp(const_net(64, 0.5), 7, 2, 1000) == 0.5
    assert ow.mlp(const_net(64, -0.75), 0, 0) == -0.75
    same = ow.seq_sim(inst, const_net(64, 0.5))
    assert (same["actions"] == plain["actions"]).all()
    cap = rng.integers(3, 9, 5)
    Sl = cap - rng.integers(0, 2, 5)
    sl = np.array([rng.integers(0, v) for v in Sl])
    inst = synth.make_owmr(400, 5, seed=4, demand="small", s_loc=sl, S_loc=Sl, cap=cap, s=20,
                           S=90)
    less = ow.seq_sim(inst, const_net(64, -0.75))
    shifted = synth.make_owmr(400, 5, seed=4, demand="small", s_loc=sl, S_loc=Sl - 1, cap=cap,
                              s=20, S=90, x0r=Sl)
    assert (less["actions"] == ow.seq_sim(shifted)["actions"]).all()
    assert less["q"].sum() < ow.seq_sim(inst)["q"].sum()


def test_network_within_fp32_bound_of_fp64():
    """z in FP32 (fixed order) against an FP64 evaluation of the same BF16
    weights; the bound is the standard gamma_n bound for n-term dot products
    propagated through the layers (relu is 1-Lipschitz)."""
    H = 128
    net = synth.make_owmr_net(H, seed=2, std=0.2)
    f = lambda a: synth.bf16_to_f32(np.asarray(a)).astype(np.float64)
    W1, b1, W2, b2, w3, b3 = f(net.W1).reshape(3, H), f(net.b1), f(net.W2).reshape(H, H), \
        f(net.b2), f(net.w3), f(net.b3)[0]
    u = 2.0 ** -24
    g = lambda n: n * u / (1 - n * u)
    worst = 0.0
    for y, d, e in [(y, d, e) for y in range(0, 40, 3) for d in range(4) for e in (1, 777, 32767)]:
        gf = e / 4096.0
        a1 = b1 + W1[0] * y + W1[1] * d + W1[2] * gf
        h1 = np.maximum(a1, 0)
        e1 = g(4) * (np.abs(b1) + np.abs(W1[0] * y) + np.abs(W1[1] * d) + np.abs(W1[2] * gf))
        a2 = b2 + h1 @ W2
        h2 = np.maximum(a2, 0)
        e2 = g(H + 1) * (np.abs(b2) + (np.abs(h1) + e1) @ np.abs(W2)) + e1 @ np.abs(W2)
        z64 = b3 + h2 @ w3
        ez = g(H + 1) * (abs(b3) + (np.abs(h2) + e2) @ np.abs(w3)) + e2 @ np.abs(w3)
        z32 = ow.mlp(net, y, d, e)
        assert abs(z32 - z64) <= ez * 1.0001 + 1e-30, (y, d, e, z32, z64, ez)
        worst = max(worst, abs(z32 - z64) / max(ez, 1e-30))
        # a dropped bias or a skipped relu is far outside the bound
        assert abs((z64 - b3) - z32) > ez or abs(b3) <= ez
    assert worst < 1.0


def test_network_output_is_one_chain_from_the_bias():
    """The FP32 order of the network's output layer, pinned by a case whose
    rounding has a closed form: with h2_j = 1 for every unit (W2 = 0, b2 = 1)
    and w3 = 1, b3 = 2^24, a single fma chain starting from b3 rounds every
    step back to 2^24 (ties to even), so z = 2^24 exactly; summing the H ones
    in groups first, or adding b3 last, gives 2^24 + H."""
    H = 64
    bf = lambda v: synth.f32_to_bf16(np.asarray(v, np.float32))
    net = synth.OwmrNet(H, bf(np.zeros((3, H))), bf(np.zeros(H)), bf(np.zeros((H, H))),
                        bf(np.ones(H)), bf(np.ones(H)), bf([2.0 ** 24]))
    assert ow.mlp(net, 5, 1, 3) == 2.0 ** 24
    # increasing j: w3_0 = 2^24 first, then the ones vanish; decreasing j would
    # give (H - 1) + 2^24, which rounds to 2^24 + H
    w3 = np.ones(H)
    w3[0] = 2.0 ** 24
    net = synth.OwmrNet(H, bf(np.zeros((3, H))), bf(np.zeros(H)), bf(np.zeros((H, H))),
                        bf(np.ones(H)), bf(w3), bf([0.0]))
    assert ow.mlp(net, 5, 1, 3) == 2.0 ** 24


def test_literal_fixed_point_prop1_random():
    """Prop. 1 for a partition by retailers: the first step where alpha^k
    differs from the sequential path moves strictly forward with k (its owner
    sees the correct state there), so the iteration reaches the sequential path
    within T + 1 passes (every case of the family, with and without Theorem
    B.1's condition, with a network, with random demand)."""
    rng = np.random.default_rng(21)
    net = synth.make_owmr_net(64, seed=9)
    for trial in range(40):
        N = int(rng.integers(1, 7))
        inst = random_inst(rng, int(rng.integers(1, 70)), N, theorem=bool(trial % 2))
        P = int(rng.integers(1, N + 1))
        proc = rng.permutation(np.arange(N) % P)
        for nn in (None, net) if trial % 4 == 0 else (None,):
            seq = ow.seq_sim(inst, nn)["actions"]
            out = ow.picard_literal(inst, nn, proc, record=True)
            assert out["converged"] and (out["actions"] == seq).all()
            assert out["iters"] <= inst.T + 1
            front = [int(np.argmax(it != seq)) if (it != seq).any() else inst.T
                     for it in out["iterates"]]
            assert all(b > a or b == inst.T for a, b in zip(front, front[1:]))


def first_exact(iterates, seq):
    k = len(iterates)
    while k > 0 and (iterates[k - 1] == seq).all():
        k -= 1
    return k + 1


def test_theorem_b1_replenishment_bound():
    """Theorem B.1: with s >= every c_n and x0 > s, the cache equals the
    sequential path after at most 2R + 1 passes counted from an empty cache
    (R = replenishments of the sequential path), and after one pass when
    R = 0; the returned pass count adds the confirming pass.  The bound is
    attained on some instances."""
    rng = np.random.default_rng(5)
    hit = 0
    for trial in range(300):
        N = int(rng.integers(1, 6))
        inst = random_inst(rng, int(rng.integers(1, 60)), N, theorem=True)
        P = int(rng.integers(1, N + 1))
        proc = rng.permutation(np.arange(N) % P)
        seq = ow.seq_sim(inst)
        out = ow.picard_literal(inst, None, proc, record=True)
        fe = first_exact(out["iterates"], seq["actions"])
        assert fe <= 2 * seq["R"] + 1, (fe, seq["R"])
        if seq["R"] == 0:
            assert fe == 1
        assert out["iters"] == fe + 1 if fe < out["iters"] else out["iters"] == fe
        hit += fe == 2 * seq["R"] + 1 and seq["R"] > 0
    assert hit > 0


def test_single_processor_is_sequential():
    rng = np.random.default_rng(8)
    net = synth.make_owmr_net(64, seed=3)
    for trial in range(10):
        inst = random_inst(rng, int(rng.integers(1, 200)), int(rng.integers(1, 6)), theorem=False)
        for nn in (None, net):
            out = ow.picard_literal(inst, nn, np.zeros(inst.N, np.int32), record=True)
            assert out["iters"] == (2 if inst.T else 1)
            assert (out["iterates"][0] == ow.seq_sim(inst, nn)["actions"]).all()


def test_walk_equals_literal_every_pass():
    """The prefix/walk organisation gives alpha^k of the literal iteration for
    every k, the same final state and statistics as the sequential path, and
    makes at most as many network calls (T in the first pass)."""
    rng = np.random.default_rng(31)
    net = synth.make_owmr_net(64, seed=4)
    for trial in range(30):
        N = int(rng.integers(1, 8))
        inst = random_inst(rng, int(rng.integers(0, 90)), N, theorem=bool(trial % 3))
        P = int(rng.integers(1, N + 1))
        proc = rng.permutation(np.arange(N) % P)
        init = None
        if trial % 5 == 4:
            init = (2 * rng.integers(0, 4, inst.T) + rng.integers(0, 2, inst.T)).astype(np.int32)
        for nn in (None, net) if trial % 3 == 0 else (None,):
            lit = ow.picard_literal(inst, nn, proc, alpha_init=init, record=True)
            wk = ow.picard_walk(inst, nn, proc, alpha_init=init, record=True)
            assert lit["iters"] == wk["iters"]
            assert (lit["iterates"] == wk["iterates"]).all()
            seq = ow.seq_sim(inst, nn)
            assert (wk["x_final"] == seq["x_final"]).all()
            assert (wk["R"], wk["lost"], wk["shipped"]) == (seq["R"], seq["lost"], seq["shipped"])
            if nn is not None:
                assert inst.T <= wk["evals"] <= lit["evals"] or inst.T == 0


def test_warm_start_and_not_converged():
    rng = np.random.default_rng(12)
    inst = random_inst(rng, 200, 5)
    proc = np.arange(5, dtype=np.int32)
    seq = ow.seq_sim(inst)["actions"]
    assert ow.picard_walk(inst, None, proc, alpha_init=seq)["iters"] == 1
    full = ow.picard_walk(inst, None, proc)
    if full["iters"] > 2:
        cut = ow.picard_walk(inst, None, proc, max_iters=full["iters"] - 1)
        assert not cut["converged"]


def test_invalid_inputs():
    inst = synth.make_owmr(10, 2, seed=0)
    bad = synth.make_owmr(10, 2, seed=0)
    bad.Sl = np.array([30, 20], np.int32)  # S_n above c_n
    with pytest.raises(ValueError):
        ow.seq_sim(bad)
    bad = synth.make_owmr(10, 2, seed=0)
    bad.S = bad.s
    with pytest.raises(ValueError):
        ow.seq_sim(bad)
    with pytest.raises(ValueError):
        ow.picard_walk(inst, None, np.array([0, -1], np.int32))


def test_window_fixed_point_and_walk_equals_literal():
    """max_steps window (Appendix A.3): every window reaches the sequential
    path; the walk gives the literal iteration's iterates pass by pass; a
    window covering the horizon gives the unwindowed iterates."""
    rng = np.random.default_rng(41)
    net = synth.make_owmr_net(64, seed=6)
    for trial in range(30):
        N = int(rng.integers(1, 7))
        inst = random_inst(rng, int(rng.integers(1, 80)), N, theorem=bool(trial % 2))
        P = int(rng.integers(1, N + 1))
        proc = rng.permutation(np.arange(N) % P)
        nn = net if trial % 3 == 0 else None
        seq = ow.seq_sim(inst, nn)["actions"]
        for W in (1, 2, 7, int(rng.integers(1, inst.T + 2))):
            lit = ow.picard_literal(inst, nn, proc, record=True, window=W)
            wk = ow.picard_walk(inst, nn, proc, record=True, window=W)
            assert lit["converged"] and (lit["actions"] == seq).all()
            assert lit["iters"] == wk["iters"] and (lit["iterates"] == wk["iterates"]).all()
        full = ow.picard_literal(inst, nn, proc, record=True)
        big = ow.picard_literal(inst, nn, proc, record=True, window=inst.T)
        assert full["iters"] == big["iters"] and (full["iterates"] == big["iterates"]).all()


@pytest.mark.parametrize("T,W", [(1, 1), (10, 3), (64, 8), (100, 7), (99, 100)])
def test_window_pass_count_closed_form(T, W):
    """One processor on a path whose every action is nonzero (unit demand,
    stores reorder up to S_n whenever below it): pass 1 writes the first
    window, pass 2 confirms it and moves on, so the iteration takes exactly
    2 ceil(T / W) passes, and alpha^(2j-1) holds the sequential path on
    [0, min(jW, T)) and zeros after it."""
    cap = np.array([9, 6, 8])
    inst = synth.make_owmr(T, 3, seed=T + W, demand="unit", s_loc=cap - 1, S_loc=cap, cap=cap,
                           s=20, S=200)
    seq = ow.seq_sim(inst)["actions"]
    assert (seq > 0).all()
    out = ow.picard_walk(inst, None, np.zeros(3, np.int32), record=True, window=W)
    assert out["iters"] == 2 * -(-T // W)
    for j in range(1, -(-T // W) + 1):
        it = out["iterates"][2 * j - 2]
        e = min(j * W, T)
        assert (it[:e] == seq[:e]).all() and (it[e:] == 0).all()
