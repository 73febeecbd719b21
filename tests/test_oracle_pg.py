"""Pins for the FP64 policy-gradient oracle (oracle/pg.py): central finite
differences of the surrogate and torch autograd of an independently written
surrogate.  CPU only."""
import numpy as np
import torch

import oracle
from oracle import pg
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.synth import Policy


def _case(T=1500, N=8, K=12, R=6, seed=0):
    inst = synth.make_instance(T, N, K, R, seed=seed, stock="poisson", fill=0.8)
    mlp = synth.make_mlp(N, R, seed=seed)
    pol = Policy("gumbel", mlp=mlp, seed=1234 + seed, traj=2)
    act = oracle.seq_sim(inst, pol)["actions"]
    return inst, mlp, act


def test_stock_before_matches_replay():
    inst, mlp, act = _case(T=400)
    S = pg.stock_before(inst, act)
    x = inst.x0.astype(np.int64).copy()
    for t in range(inst.T):
        np.testing.assert_array_equal(S[t], x[inst.prod[t]])
        if act[t] >= 0:
            x[inst.prod[t], act[t]] -= 1


def test_returns_to_go_closed_form():
    inst, mlp, act = _case(T=300)
    G = pg.returns_to_go(inst, act)
    c = [int(inst.cost[inst.reg[t], act[t]]) if act[t] >= 0 else 0 for t in range(inst.T)]
    for t in (0, 1, 17, inst.T - 1):
        assert G[t] == -sum(c[t:])


def test_pg_gradient_vs_central_differences():
    """Central differences of J in FP64, trajectory held fixed, on 80 random
    coordinates across all five parameter tensors.  A step can straddle a ReLU
    kink (bias coordinates shift every order's pre-activation) and very small
    steps meet FP64 cancellation in J, so each coordinate is differenced with two
    steps and must agree with the analytic value at one of them."""
    inst, mlp, act = _case(T=600)
    P = pg.bf16_params_f64(mlp)
    J0, g = pg.surrogate(inst, P, act)
    assert np.isfinite(J0) and J0 != 0.0
    rng = np.random.default_rng(0)
    best, an = [], []
    for _ in range(80):
        name = pg.PARAMS[int(rng.integers(0, 5))]
        if name == "E":  # only regions that occur carry gradient; pick one that does
            i = (int(inst.reg[int(rng.integers(0, inst.T))]), int(rng.integers(0, 16)))
        else:
            i = tuple(int(rng.integers(0, d)) for d in P[name].shape)
        ests = []
        for h0 in (1e-5, 1e-6):
            h = h0 * max(1.0, abs(P[name][i]))
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][i] += h
            Pm[name][i] -= h
            Jp, _ = pg.surrogate(inst, Pp, act, grad=False)
            Jm, _ = pg.surrogate(inst, Pm, act, grad=False)
            ests.append((Jp - Jm) / (2 * h))
        a = g[name][i]
        best.append(min(ests, key=lambda e: abs(e - a)))
        an.append(a)
    best, an = np.array(best), np.array(an)
    assert np.linalg.norm(best - an) / np.linalg.norm(best) < 1e-6
    assert np.all(np.abs(best - an) <= 1e-4 * np.abs(best) + 1e-6 * np.abs(best).max())


def test_pg_gradient_vs_torch_autograd():
    """Full gradient against torch autograd (FP64) of the same surrogate written
    with torch ops: log_softmax over the feasible set, returns-to-go weights."""
    inst, mlp, act = _case(T=2500, N=16, K=20, R=9, seed=3)
    P = pg.bf16_params_f64(mlp)
    J0, g = pg.surrogate(inst, P, act)
    th = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in P.items()}
    # state along the trajectory by plain replay
    x = inst.x0.astype(np.int64).copy()
    rows = np.zeros((inst.T, inst.N), np.int64)
    for t in range(inst.T):
        rows[t] = x[inst.prod[t]]
        if act[t] >= 0:
            x[inst.prod[t], act[t]] -= 1
    c = np.array([inst.cost[inst.reg[t], act[t]] if act[t] >= 0 else 0 for t in range(inst.T)])
    Gt = torch.tensor(-np.cumsum(c[::-1])[::-1].copy(), dtype=torch.float64)
    S = torch.tensor(rows)
    feas = S > 0
    keep = torch.tensor(act >= 0) & (feas.sum(1) >= 2)
    reg = torch.tensor(inst.reg.astype(np.int64))
    cost = torch.tensor(inst.cost.astype(np.float64))
    feats = torch.cat([cost[reg] / 128.0, torch.clamp(S, max=32).double() / 32.0, th["E"][reg]], 1)
    z = feats @ th["W1"] + th["b1"]
    s = torch.relu(z) @ th["W2"] + th["b2"]
    s = torch.where(feas, s, torch.full_like(s, -torch.inf))
    lp = torch.log_softmax(s, dim=1)
    a = torch.tensor(np.maximum(act, 0).astype(np.int64))
    chosen = lp.gather(1, a[:, None])[:, 0]
    Jt = torch.where(keep, chosen * Gt, torch.zeros_like(Gt)).sum()
    Jt.backward()
    assert abs(Jt.item() - J0) <= 1e-9 * abs(J0)
    for k in pg.PARAMS:
        want = th[k].grad.numpy()
        err = np.linalg.norm(g[k] - want) / max(np.linalg.norm(want), 1e-30)
        assert err < 1e-9, (k, err)
