"""Policy gradient on the GPU (pic_policy_grad and its torch.autograd.Function)
against the FP64 oracle (oracle/pg.py: the surrogate and its gradient, itself
pinned by finite differences and torch autograd), against FP64 central
differences directly, and against torch autograd of a surrogate written here.
Paths simulated inside the call must equal the oracle's sequential paths
bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import paper_2406_01939_b300 as pic
from oracle import pg
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.reinforce import Reinforce, flat_from_mlp, split_flat
from paper_2406_01939_b300.session import DeviceBatch
from paper_2406_01939_b300.synth import Policy

pytestmark = pytest.mark.gpu

NAMES = ("W1", "b1", "W2", "b2", "E")
TOL = 1e-3


def case(seed, Ts, N, K, R, fill=0.8):
    insts = [synth.make_instance(int(T), N, K, R, seed=100 * seed + b, stock="poisson", fill=fill)
             for b, T in enumerate(Ts)]
    mlp = synth.make_mlp(N, R, seed=seed)
    pols = [Policy("gumbel", mlp=mlp, seed=5000 + seed, traj=b) for b in range(len(Ts))]
    return insts, mlp, pols


def oracle_batch(insts, pols, params, acts=None):
    J, gsum = 0.0, None
    paths = []
    for b, (inst, pol) in enumerate(zip(insts, pols)):
        a = oracle.seq_sim(inst, pol)["actions"] if acts is None else acts[b]
        paths.append(a)
        Jb, gb = pg.surrogate(inst, params, a)
        J += Jb
        gsum = gb if gsum is None else {k: gsum[k] + gb[k] for k in gsum}
    return J, gsum, paths


def run_gpu(insts, pols, mlp, master=None, num_chunks=16):
    db = DeviceBatch(insts)
    N, R = insts[0].N, insts[0].R
    rf = Reinforce(db, [p.kind for p in pols], [p.seed for p in pols], [p.traj for p in pols], R,
                   num_chunks=num_chunks)
    m = flat_from_mlp(mlp) if master is None else master
    acts = torch.empty(db.T, dtype=torch.int8, device="cuda")
    J, res = rf.objective(m, actions_out=acts)
    g = torch.empty_like(m)
    J2 = rf.gradient(m, acts, g)
    return db, rf, m, acts, J, J2, split_flat(g.cpu().double(), N, R)


def assert_close_grad(got, want, tol=TOL, outlier_frac=0.0):
    """Norm-wise relative error <= tol overall and per tensor, and elementwise
    |err| <= tol * max|want| for all but outlier_frac of each tensor's entries."""
    num = sum(float(((got[k].numpy() - want[k]) ** 2).sum()) for k in NAMES)
    den = sum(float((want[k] ** 2).sum()) for k in NAMES)
    assert np.sqrt(num / den) <= tol, np.sqrt(num / den)
    for k in NAMES:
        w, g = want[k], got[k].numpy()
        if np.abs(w).max() == 0:
            assert np.abs(g).max() == 0, k
            continue
        rel = np.linalg.norm(g - w) / np.linalg.norm(w)
        assert rel <= tol, (k, rel)
        bad = np.abs(g - w) > tol * np.abs(w).max()
        assert bad.sum() <= outlier_frac * bad.size, (k, int(bad.sum()))


@pytest.mark.parametrize("N", [8, 16, 64])
def test_paths_objective_and_gradient_match_oracle(N):
    insts, mlp, pols = case(N, [1800, 2500, 900], N, K=24, R=11)
    db, rf, m, acts, J, J2, g = run_gpu(insts, pols, mlp)
    P = pg.bf16_params_f64(mlp)
    Jw, gw, paths = oracle_batch(insts, pols, P)
    a = acts.cpu().numpy()
    for b in range(len(insts)):
        np.testing.assert_array_equal(db.split(a)[b], paths[b])
    # J2 comes from the gradient kernel (tensor cores, split BF16 products)
    assert abs(J - Jw) <= 1e-5 * abs(Jw) and abs(J2 - Jw) <= 1e-5 * abs(Jw)
    assert_close_grad(g, gw)


def test_long_products_walked_in_pieces():
    """Products with more than 1,024 orders (K = 3 over 9,000 and 5,000 orders):
    their stock features are walked in pieces from per-piece action counts; the
    objective and gradient equal the oracle's, and so do the paths."""
    insts, mlp, pols = case(12, [9000, 5000], 32, K=3, R=7, fill=1.2)
    assert min(np.bincount(i.prod).max() for i in insts) > 2 * 1024
    db, rf, m, acts, J, J2, g = run_gpu(insts, pols, mlp)
    P = pg.bf16_params_f64(mlp)
    Jw, gw, paths = oracle_batch(insts, pols, P)
    a = acts.cpu().numpy()
    for b in range(len(insts)):
        np.testing.assert_array_equal(db.split(a)[b], paths[b])
    assert abs(J - Jw) <= 1e-5 * abs(Jw) and abs(J2 - Jw) <= 1e-5 * abs(Jw)
    assert_close_grad(g, gw)


def test_gradient_vs_fp64_central_differences():
    """Central differences of the FP64 objective at sampled coordinates of every
    parameter tensor; each coordinate tried with two steps (a step can cross a
    ReLU kink) and the closer estimate kept."""
    insts, mlp, pols = case(3, [1500, 1100], 16, K=20, R=9)
    _, _, _, acts, _, _, g = run_gpu(insts, pols, mlp)
    P = pg.bf16_params_f64(mlp)
    paths = [oracle.seq_sim(i, p)["actions"] for i, p in zip(insts, pols)]

    def Jof(params):
        return sum(pg.surrogate(i, params, a, grad=False)[0] for i, a in zip(insts, paths))

    rng = np.random.default_rng(1)
    fd, an = [], []
    for _ in range(48):
        name = NAMES[int(rng.integers(0, 5))]
        if name == "E":
            i = (int(insts[0].reg[int(rng.integers(0, insts[0].T))]), int(rng.integers(0, 16)))
        else:
            i = tuple(int(rng.integers(0, d)) for d in P[name].shape)
        a_val = float(g[name][i])
        ests = []
        for h0 in (1e-5, 1e-6):
            h = h0 * max(1.0, abs(P[name][i]))
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][i] += h
            Pm[name][i] -= h
            ests.append((Jof(Pp) - Jof(Pm)) / (2 * h))
        fd.append(min(ests, key=lambda e: abs(e - a_val)))
        an.append(a_val)
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd - an) / np.linalg.norm(fd) <= TOL
    assert np.all(np.abs(fd - an) <= TOL * np.abs(fd).max())


def torch_surrogate(insts, paths, P):
    """REINFORCE surrogate written with torch ops (FP64, autograd)."""
    W1, b1, W2, b2, E = (P[k] for k in NAMES)
    J = torch.zeros((), dtype=torch.float64)
    for inst, a in zip(insts, paths):
        N = inst.N
        x = inst.x0.astype(np.int64).copy()
        rows, acts, G, masks = [], [], [], []
        costs = np.where(a >= 0, inst.cost[inst.reg, np.maximum(a, 0)], 0).astype(np.int64)
        suffix = np.cumsum(costs[::-1])[::-1]
        for t in range(inst.T):
            k = inst.prod[t]
            s = x[k].copy()
            if a[t] >= 0:
                x[k, a[t]] -= 1
            if a[t] < 0 or (s > 0).sum() < 2:
                continue
            rows.append((inst.reg[t], np.minimum(s, 32) / 32.0))
            acts.append(a[t])
            G.append(-float(suffix[t]))
            masks.append(s > 0)
        if not rows:
            continue
        r = torch.tensor(np.array([q[0] for q in rows], dtype=np.int64))
        f = torch.tensor(np.stack([q[1] for q in rows]))
        c = torch.tensor(inst.cost.astype(np.float64))[r] / 128.0
        xin = torch.cat([c, f, E[r]], dim=1)
        sc = torch.relu(xin @ W1 + b1) @ W2 + b2
        sc = sc.masked_fill(~torch.tensor(np.stack(masks)), float("-inf"))
        lp = torch.log_softmax(sc, dim=1)[torch.arange(len(acts)),
                                          torch.tensor(np.array(acts, dtype=np.int64))]
        J = J + (lp * torch.tensor(G)).sum()
    return J


def test_gradient_vs_torch_autograd():
    insts, mlp, pols = case(7, [2200, 1300], 32, K=30, R=12)
    _, _, _, acts, J, _, g = run_gpu(insts, pols, mlp)
    P = {k: torch.tensor(v, requires_grad=True) for k, v in pg.bf16_params_f64(mlp).items()}
    paths = [oracle.seq_sim(i, p)["actions"] for i, p in zip(insts, pols)]
    Jt = torch_surrogate(insts, paths, P)
    Jt.backward()
    assert abs(J - float(Jt.detach())) <= 1e-5 * abs(float(Jt.detach()))
    assert_close_grad(g, {k: P[k].grad.numpy() for k in NAMES})


def test_autograd_function_and_given_paths():
    """The autograd.Function's backward returns the kernel gradient scaled by the
    upstream gradient; a call on given paths reproduces the simulated call."""
    insts, mlp, pols = case(9, [1700, 800, 1200], 8, K=16, R=7)
    db = DeviceBatch(insts)
    rf = Reinforce(db, ["gumbel"] * 3, [p.seed for p in pols], [p.traj for p in pols], 7, num_chunks=8)
    m = flat_from_mlp(mlp).requires_grad_(True)
    J = rf(m)
    (3.0 * J).backward()
    g_direct = torch.empty_like(m)
    Jd = rf.gradient(m.detach(), rf.last_actions, g_direct)
    assert abs(float(J.detach()) - Jd) <= 1e-5 * abs(Jd)
    torch.testing.assert_close(m.grad, 3.0 * g_direct, rtol=1e-6, atol=0)
    # masters that are not BF16 values: the gradient is taken at the rounded values
    m2 = (m.detach() * (1 + 1e-4)).contiguous()
    acts2 = torch.empty(db.T, dtype=torch.int8, device="cuda")
    rf.objective(m2, actions_out=acts2)
    g2 = torch.empty_like(m2)
    rf.gradient(m2, acts2, g2)
    rounded = synth.MLPParams(*[synth.f32_to_bf16(v.cpu().numpy()) for v in
                                split_flat(m2, 8, 7).values()])
    Jw, gw, paths = oracle_batch(insts, [Policy("gumbel", mlp=rounded, seed=p.seed, traj=p.traj)
                                         for p in pols], pg.bf16_params_f64(rounded))
    a2 = acts2.cpu().numpy()
    for b in range(3):
        np.testing.assert_array_equal(db.split(a2)[b], paths[b])
    assert_close_grad(split_flat(g2.cpu().double(), 8, 7), gw)


def test_tensor_core_tiles_in_the_simulation():
    """Gumbel paths simulated with the tensor-core tiles (PIC_FLAG_TC) are the
    oracle's; the gradient along them is unchanged."""
    insts, mlp, pols = case(12, [5000, 7000], 32, K=4, R=8, fill=1.5)
    db = DeviceBatch(insts)
    rf = Reinforce(db, ["gumbel"] * 2, [p.seed for p in pols], [p.traj for p in pols], 8,
                   num_chunks=3, flags=pic.PIC_FLAG_TC | pic.PIC_FLAG_NO_SAT)
    m = flat_from_mlp(mlp)
    acts = torch.empty(db.T, dtype=torch.int8, device="cuda")
    J, res = rf.objective(m, actions_out=acts)
    assert res.tc_decisions > 0
    a = acts.cpu().numpy()
    for b, (inst, pol) in enumerate(zip(insts, pols)):
        np.testing.assert_array_equal(db.split(a)[b], oracle.seq_sim(inst, pol)["actions"])


@pytest.mark.parametrize("N", [16, 64])
def test_tensor_core_and_cuda_core_gradients_agree(N):
    """The tcgen05 gradient kernel (default) and the FP32 CUDA-core kernel
    (PIC_FLAG_NO_TC) give the same gradient along the same paths."""
    insts, mlp, pols = case(40 + N, [3000, 2000, 4100], N, K=30, R=13)
    db = DeviceBatch(insts)
    m = flat_from_mlp(mlp)
    rf = Reinforce(db, ["gumbel"] * 3, [p.seed for p in pols], [p.traj for p in pols], 13, num_chunks=8)
    rf_cc = Reinforce(db, ["gumbel"] * 3, [p.seed for p in pols], [p.traj for p in pols], 13, num_chunks=8,
                      flags=pic.PIC_FLAG_NO_TC)
    acts = torch.empty(db.T, dtype=torch.int8, device="cuda")
    rf.objective(m, actions_out=acts)
    g_tc, g_cc = torch.empty_like(m), torch.empty_like(m)
    J_tc = rf.gradient(m, acts, g_tc)
    J_cc = rf_cc.gradient(m, acts, g_cc)
    assert abs(J_tc - J_cc) <= 1e-5 * abs(J_cc)
    a = split_flat(g_tc.cpu().double(), N, 13)
    b = split_flat(g_cc.cpu().double(), N, 13)
    assert_close_grad(a, {k: v.numpy() for k, v in b.items()})


def test_infeasible_paths_rejected():
    insts, mlp, pols = case(4, [300, 400], 8, K=6, R=5)
    db = DeviceBatch(insts)
    rf = Reinforce(db, ["gumbel"] * 2, [1, 2], [0, 1], 5, num_chunks=4)
    m = flat_from_mlp(mlp)
    bad = np.zeros(db.T, np.int8)  # every order to warehouse 0: runs out of stock
    with pytest.raises(pic.PicError) as e:
        rf.objective(m, actions=torch.from_numpy(bad).cuda())
    assert e.value.status == pic.PIC_ERR_INVALID_ARG and "feasible" in str(e.value)
    out_of_range = np.full(db.T, 9, np.int8)
    with pytest.raises(pic.PicError) as e:
        rf.objective(m, actions=torch.from_numpy(out_of_range).cuda())
    assert e.value.status == pic.PIC_ERR_INVALID_ARG


def test_full_size_trajectory_gradient():
    """One trajectory of the policy-gradient shape (T=2^20, N=64, K=10,000,
    R=1,000, Gumbel MLP): the path's first 2^18 orders equal the oracle's
    sequential simulation of those orders (a prefix of the path depends only on
    the orders before it), the whole path equals the GPU sequential simulator's,
    and the gradient matches the FP64 oracle gradient along the GPU paths."""
    insts, mlp = synth.pg_large(0, B=1)
    inst = insts[0]
    pol = Policy("gumbel", mlp=mlp, seed=77, traj=0)
    db, rf, m, acts, J, J2, g = run_gpu([inst], [pol], mlp, num_chunks=0)
    a = acts.cpu().numpy()
    Tp = 1 << 18
    pre = synth.Instance(Tp, inst.N, inst.K, inst.R, inst.prod[:Tp].copy(), inst.reg[:Tp].copy(),
                         inst.x0, inst.cost, inst.lam)
    np.testing.assert_array_equal(a[:Tp], oracle.seq_sim(pre, pol)["actions"])
    seq = db.simulate([pol], "sequential")
    np.testing.assert_array_equal(seq["actions"].cpu().numpy(), a)
    Jw, gw = pg.surrogate(inst, pg.bf16_params_f64(mlp), a)
    assert abs(J - Jw) <= 1e-5 * abs(Jw)
    # 2.7e8 hidden pre-activations: a few lie within FP32 rounding of 0, where the
    # FP32 kernel and the FP64 oracle take the ReLU on opposite sides; each such
    # order moves a handful of entries (0.1% allowance) but not the norms
    assert_close_grad(g, gw, outlier_frac=1e-3)
