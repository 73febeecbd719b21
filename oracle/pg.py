"""FP64 policy-gradient oracle -- TEST INFRASTRUCTURE (see oracle/__init__.py).

The paper trains its FO policy by policy gradient over simulated roll-outs
(Sec. 4.2, Table 2).  This module states the gradient that the CUDA path
computes, in plain numpy FP64, for a fixed simulated trajectory:

    J(theta) = sum_t  log pi_theta(a_t | s_t) * G_t,      G_t = - sum_{t' >= t} c_{t'}

with c_t = cost[r_t][a_t] for fulfilled orders and 0 for a^phi, pi_theta the
softmax of the MLP scores over the feasible set F_t = {n : stock_n > 0}, and the
trajectory (s_t, a_t, G_t) held fixed (the REINFORCE surrogate).  Steps with
a_t = a^phi or |F_t| <= 1 contribute nothing (log pi = 0 when one node is
feasible).  Parameters are the BF16 values taken exactly as FP64 numbers.

Pins: central finite differences of J (FP64) and torch autograd of an
independently written surrogate (tests/test_oracle_pg.py).
"""
from __future__ import annotations

import numpy as np

PARAMS = ("W1", "b1", "W2", "b2", "E")


def bf16_params_f64(mlp):
    out = {}
    for k in PARAMS:
        b = np.ascontiguousarray(getattr(mlp, k), np.uint16).astype(np.uint32) << 16
        out[k] = b.view(np.float32).astype(np.float64)
    return out


def stock_before(inst, actions):
    """Stock row of each order's product just before the order (T x N int64):
    x0[k_t] minus the fulfilled actions of product k_t at earlier times."""
    T, N = inst.T, inst.N
    prod = np.asarray(inst.prod, np.int64)
    act = np.asarray(actions, np.int64)
    onehot = np.zeros((T, N), np.int64)
    f = act >= 0
    onehot[np.flatnonzero(f), act[f]] = 1
    order = np.argsort(prod, kind="stable")
    cs = np.cumsum(onehot[order], axis=0) - onehot[order]  # exclusive prefix, all products
    # subtract the running total at each product's first position
    p_sorted = prod[order]
    starts = np.flatnonzero(np.r_[True, p_sorted[1:] != p_sorted[:-1]])
    seg_id = np.cumsum(np.r_[True, p_sorted[1:] != p_sorted[:-1]]) - 1
    cs = cs - cs[starts][seg_id]
    used = np.empty_like(cs)
    used[order] = cs
    return np.asarray(inst.x0, np.int64)[prod] - used


def returns_to_go(inst, actions):
    act = np.asarray(actions, np.int64)
    c = np.where(act >= 0, np.asarray(inst.cost, np.int64)[inst.reg, np.maximum(act, 0)], 0)
    return -np.cumsum(c[::-1])[::-1]


def surrogate(inst, params, actions, grad=True, batch=4096):
    """Return (J, grads) in FP64.  params: dict of FP64 arrays (see bf16_params_f64)."""
    N = inst.N
    W1, b1, W2, b2, E = (params[k] for k in PARAMS)
    S = stock_before(inst, actions)
    G = returns_to_go(inst, actions).astype(np.float64)
    act = np.asarray(actions, np.int64)
    cost = np.asarray(inst.cost, np.float64)
    reg = np.asarray(inst.reg, np.int64)
    J = 0.0
    gr = {k: np.zeros_like(v) for k, v in params.items()} if grad else None
    for lo in range(0, inst.T, batch):
        hi = min(lo + batch, inst.T)
        s_ = S[lo:hi]
        a_ = act[lo:hi]
        F = s_ > 0
        use = (a_ >= 0) & (F.sum(axis=1) >= 2)
        if not use.any():
            continue
        idx = np.flatnonzero(use)
        r = reg[lo:hi][idx]
        a = a_[idx]
        Fm = F[idx]
        x = np.concatenate([cost[r] / 128.0, np.minimum(s_[idx], 32) / 32.0, E[r]], axis=1)
        z = x @ W1 + b1
        h = np.maximum(z, 0.0)
        sc = h @ W2 + b2
        masked = np.where(Fm, sc, -np.inf)
        mx = masked.max(axis=1, keepdims=True)
        lse = mx[:, 0] + np.log(np.exp(masked - mx).sum(axis=1))
        logp = sc[np.arange(len(a)), a] - lse
        g_t = G[lo:hi][idx]
        J += float((logp * g_t).sum())
        if grad:
            p = np.where(Fm, np.exp(masked - lse[:, None]), 0.0)
            ds = -p
            ds[np.arange(len(a)), a] += 1.0
            ds *= g_t[:, None]
            gr["b2"] += ds.sum(axis=0)
            gr["W2"] += h.T @ ds
            dz = (ds @ W2.T) * (z > 0)
            gr["b1"] += dz.sum(axis=0)
            gr["W1"] += x.T @ dz
            np.add.at(gr["E"], r, dz @ W1[2 * N:].T)
    return J, gr
