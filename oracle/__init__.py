"""CPU oracle for Picard-iteration FO policy simulation -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA implementation:
the arithmetic lives in ``fo_oracle.c`` (plain C, compiled with
``-ffp-contract=off``) and, for the policy gradient, in ``pg.py`` (numpy FP64).

Inputs are duck-typed: an instance needs attributes T, N, K, R, prod, reg, x0,
cost, lam; a policy needs kind ('greedy' | 'dual' | 'mlp' | 'gumbel'), mlp (with
W1, b1, W2, b2, E as BF16 uint16 arrays and H), seed and traj.

Parity status per function (see each docstring for its pins): every function
here is pinned by tests under ``tests/test_oracle_*.py``; none is unpinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fo_oracle.c")
_LIB = os.path.join(_HERE, "libfo_oracle.so")
_lock = threading.Lock()
_lib = None

KINDS = {"greedy": 0, "dual": 1, "mlp": 2, "gumbel": 3}
OK, ERR_ARG, ERR_NOT_CONVERGED = 0, 1, 4


def build(force: bool = False) -> str:
    """Compile fo_oracle.c (and the OWMR oracle, owmr_oracle.c) with gcc (IEEE
    FP32, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    from . import owmr
    owmr.build(force)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i32, i64, u64 = C.c_int32, C.c_int64, C.c_uint64
            common = [i32, i32, i32, i32, P, P, P, P, P, i32, i32, P, P, P, P, P, u64, i32]
            lib.orc_seq_sim.argtypes = common + [P, P, P, P]
            lib.orc_seq_sim.restype = C.c_int
            lib.orc_picard_literal.argtypes = common + [i32, i32, P, P, P, P]
            lib.orc_picard_literal.restype = C.c_int
            lib.orc_picard_chunked.argtypes = common + [i32, i32, P, P, P, P, P, P]
            lib.orc_picard_chunked.restype = C.c_int
            lib.orc_picard_windowed.argtypes = common + [i32, i64, i32, P, P, P, P, P, P]
            lib.orc_picard_windowed.restype = C.c_int
            capc = [i32, i32, i32, i32, P, P, P, P, P, P, i32]
            lib.orc_seq_sim_cap.argtypes = capc + [P, P, P, P, P]
            lib.orc_seq_sim_cap.restype = C.c_int
            lib.orc_picard_chunked_cap.argtypes = capc + [i32, i32, P, P, P, P, P, P]
            lib.orc_picard_chunked_cap.restype = C.c_int
            lib.orc_picard_partition.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, i32, i32,
                                                 P, P, P, P, P, u64, i32, P, i32, i32, P, P, P, P]
            lib.orc_picard_partition.restype = C.c_int
            lib.orc_mlp_scores.argtypes = [C.c_int, C.c_int, P, P, P, P, P, P, i32, P, P]
            lib.orc_mlp_scores.restype = None
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_philox4x32_10.restype = None
            lib.orc_uniform.argtypes = [u64, i32, i64, i32]
            lib.orc_uniform.restype = C.c_float
            lib.orc_log.argtypes = [C.c_float]
            lib.orc_log.restype = C.c_float
            lib.orc_gumbel.argtypes = [u64, i32, i64, i32]
            lib.orc_gumbel.restype = C.c_float
            lib.orc_state_before.argtypes = [i32, i32, P, P, P, i64, P]
            lib.orc_state_before.restype = C.c_int
            lib.orc_policy_call.argtypes = [i32, i32, P, P, i32, i32, P, P, P, P, P, u64, i32,
                                            P, i32, i32, i64]
            lib.orc_policy_call.restype = C.c_int
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def _args(inst, pol):
    kind = KINDS[pol.kind]
    m = pol.mlp
    keep = [
        _c(inst.prod, np.int32), _c(inst.reg, np.int32), _c(inst.x0, np.int32),
        _c(inst.cost, np.int32), _c(inst.lam, np.int32) if kind == 1 else None,
    ]
    if kind >= 2:
        mk = [_c(m.W1, np.uint16), _c(m.b1, np.uint16), _c(m.W2, np.uint16), _c(m.b2, np.uint16),
              _c(m.E, np.uint16)]
        H = int(m.H)
    else:
        mk, H = [None] * 5, 0
    keep += mk
    args = [inst.T, inst.N, inst.K, inst.R] + [_p(a) for a in keep[:5]] + [kind, H] + \
        [_p(a) for a in mk] + [int(pol.seed) & 0xFFFFFFFFFFFFFFFF, int(pol.traj)]
    return args, keep


def _cap(inst):
    cap = getattr(inst, "cap", None)
    return None if cap is None else _c(cap, np.int32)


def _cap_args(inst, pol, cap):
    kind = KINDS[pol.kind]
    if kind >= 2:
        raise ValueError("capacity: integer policies only (greedy, dual)")
    keep = [_c(inst.prod, np.int32), _c(inst.reg, np.int32), _c(inst.x0, np.int32), cap,
            _c(inst.cost, np.int32), _c(inst.lam, np.int32) if kind == 1 else None]
    return [inst.T, inst.N, inst.K, inst.R] + [_p(a) for a in keep] + [kind], keep


def seq_sim(inst, pol):
    """Sequential simulation a_t = pi(s_t, w_t), s_{t+1} = f(s_t, a_t, w_t)
    (Sec. 2 problem statement, Sec. 3 inventory dynamics; with inst.cap set, the
    Sec. 3 state (x, c) with node capacity, integer policies only, and the
    result also holds "c_final").

    Pins: brute-force argmin/argmax per step on tiny inputs, conservation
    (units shipped = x0 - x_final, = cap - c_final per node), non-negative stock
    and capacity, a^phi iff no feasible node, textbook special cases (ample
    stock => unconstrained argmin; ample capacity => the inventory-only path)."""
    lib = _load()
    cap = _cap(inst)
    if cap is not None:
        args, keep = _cap_args(inst, pol, cap)
        act = np.empty(inst.T, np.int8)
        xf = np.empty((inst.K, inst.N), np.int32)
        cf = np.empty(inst.N, np.int32)
        tc, lost = C.c_int64(0), C.c_int64(0)
        rc = lib.orc_seq_sim_cap(*args, _p(act), _p(xf), _p(cf), C.byref(tc), C.byref(lost))
        if rc != OK:
            raise ValueError(f"orc_seq_sim_cap failed rc={rc}")
        return {"actions": act, "x_final": xf, "c_final": cf, "total_cost": tc.value,
                "lost": lost.value}
    args, keep = _args(inst, pol)
    act = np.empty(inst.T, np.int8)
    xf = np.empty((inst.K, inst.N), np.int32)
    tc, lost = C.c_int64(0), C.c_int64(0)
    rc = lib.orc_seq_sim(*args, _p(act), _p(xf), C.byref(tc), C.byref(lost))
    if rc != OK:
        raise ValueError(f"orc_seq_sim failed rc={rc}")
    return {"actions": act, "x_final": xf, "total_cost": tc.value, "lost": lost.value}


def _picard(fn, inst, pol, M, max_iters, alpha_init, record, extra, args=None, keep=None):
    lib = _load()
    if args is None:
        args, keep = _args(inst, pol)
    if max_iters is None:
        max_iters = M + 1
    act = np.empty(inst.T, np.int8)
    iters = C.c_int32(0)
    its = np.empty((max_iters, inst.T), np.int8) if record else None
    ai = _c(alpha_init, np.int8)
    out = {}
    tail = [_p(ai), _p(act), C.byref(iters), _p(its)]
    if extra:
        chg = np.zeros(max_iters, np.int64)
        fst = np.zeros(max_iters, np.int64)
        tail += [_p(chg), _p(fst)]
    rc = fn(*args, int(M), int(max_iters), *tail)
    if rc not in (OK, ERR_NOT_CONVERGED):
        raise ValueError(f"picard oracle failed rc={rc}")
    k = iters.value
    out.update(actions=act, iters=k, converged=(rc == OK))
    if record:
        out["iterates"] = its[:k].copy()
    if extra:
        out["changed"] = chg[:k].copy()
        out["first_changed"] = fst[:k].copy()
    return out


def picard_literal(inst, pol, M, max_iters=None, alpha_init=None, record=False):
    """Algorithm 1 verbatim on M contiguous time blocks: every process restarts
    from s_1, evaluates pi on its block, applies feasible cached actions elsewhere.

    Pins: equals seq_sim (Prop. 1); alpha^k exact on blocks 0..k-1 after pass k
    (proof of Prop. 1); M=1 and ample stock converge in 2 passes; iteration bound
    of Sec. 3.1 for greedy; brute force over tiny instances."""
    return _picard(_load().orc_picard_literal, inst, pol, M, max_iters, alpha_init, record, False)


def picard_chunked(inst, pol, M, max_iters=None, alpha_init=None, record=False):
    """Algorithm 1 on the same blocks with the cached-prefix replay in closed form
    max(0, x0 - d) (with inst.cap set: also c = max(0, cap - q), q the cached
    actions that found inventory).  Pins: identical iterates alpha^k to
    picard_literal / picard_partition for every k on exhaustive tiny instances
    and random small ones; fixed point = seq_sim; ample capacity gives the
    inventory-only iterates."""
    cap = _cap(inst)
    if cap is not None:
        args, keep = _cap_args(inst, pol, cap)
        return _picard(_load().orc_picard_chunked_cap, inst, pol, M, max_iters, alpha_init,
                       record, True, args, keep)
    return _picard(_load().orc_picard_chunked, inst, pol, M, max_iters, alpha_init, record, True)


def picard_windowed(inst, pol, M, max_steps, max_iters=None, alpha_init=None, record=False):
    """Algorithm 1 on M contiguous blocks with the max_steps window of Appendix
    A.3 (no capacity): a pass evaluates only the blocks that start before
    w_start + max_steps; the window starts at the first changed time of the
    previous pass, or moves past the evaluated blocks after a pass without
    change; the loop returns after a pass without change that evaluated every
    block.  max_iters defaults to 2 M + 2.

    Pins: max_steps >= T gives the iterates of picard_chunked; the fixed point is
    seq_sim for every max_steps (exhaustive tiny family and random instances,
    every policy kind); with one block per window at most 2 M passes."""
    if max_iters is None:
        max_iters = 2 * M + 2
    lib = _load()
    args, keep = _args(inst, pol)
    act = np.empty(inst.T, np.int8)
    iters = C.c_int32(0)
    its = np.empty((max_iters, inst.T), np.int8) if record else None
    chg = np.zeros(max_iters, np.int64)
    fst = np.zeros(max_iters, np.int64)
    ai = _c(alpha_init, np.int8)
    rc = lib.orc_picard_windowed(*args, int(M), int(max_steps), int(max_iters), _p(ai), _p(act),
                                 C.byref(iters), _p(its), _p(chg), _p(fst))
    if rc not in (OK, ERR_NOT_CONVERGED):
        raise ValueError(f"orc_picard_windowed failed rc={rc}")
    k = iters.value
    out = {"actions": act, "iters": k, "converged": rc == OK, "changed": chg[:k].copy(),
           "first_changed": fst[:k].copy()}
    if record:
        out["iterates"] = its[:k].copy()
    return out


def picard_partition(inst, pol, proc, max_iters=None, alpha_init=None, record=False):
    """Algorithm 1 verbatim for any assignment proc[t] of time-steps to
    processes (contiguous blocks, product partitions of Sec. 3, uniform random
    assignment), with node capacity when inst.cap is set.  M = max(proc) + 1;
    max_iters defaults to T + 1 (Prop. 1).

    Pins: with proc[t] = t // L it equals picard_literal (no capacity) and
    picard_chunked (capacity) iterate by iterate; its fixed point is seq_sim
    (Prop. 1); with product partitions and a greedy / bid-price policy the cache
    is exact after at most |Q_T| + 1 passes, Q_T the nodes whose capacity the
    sequential path exhausts (Thm. 3.1); without binding capacity product
    partitions are exact after one pass."""
    lib = _load()
    cap = _cap(inst)
    pr = _c(proc, np.int32)
    M = int(pr.max()) + 1 if len(pr) else 1
    if max_iters is None:
        max_iters = inst.T + 1
    base, keep = _args(inst, pol)
    # base: T,N,K,R,prod,reg,x0,cost,lam,kind,H,W1,b1,W2,b2,E,seed,traj
    args = base[:7] + [_p(cap)] + base[7:] + [_p(pr)]
    keep = keep + [cap, pr]
    return _picard(lib.orc_picard_partition, inst, pol, M, max_iters, alpha_init, record, False,
                   args, keep)


def mlp_scores(N, mlp, cost_row, r, stock_row):
    """Fixed-order FP32 MLP scores.  Pins: agrees with an FP64 matrix product of
    the same parameters to within the FP32 accumulation bound."""
    lib = _load()
    keep = [_c(mlp.W1, np.uint16), _c(mlp.b1, np.uint16), _c(mlp.W2, np.uint16),
            _c(mlp.b2, np.uint16), _c(mlp.E, np.uint16), _c(cost_row, np.int32),
            _c(stock_row, np.int32)]
    out = np.empty(N, np.float32)
    lib.orc_mlp_scores(N, int(mlp.H), *[_p(a) for a in keep[:6]], int(r), _p(keep[6]), _p(out))
    return out


def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11).  Pin: published known-answer
    vectors (tests/golden/philox4x32_10_kat.txt)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.empty(4, np.uint32)
    lib.orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def log32(x):
    """IEEE-only FP32 natural log.  Pin: within 2 ulp of FP64 log."""
    return np.float32(_load().orc_log(float(x)))


def uniform(seed, traj, t, n):
    return np.float32(_load().orc_uniform(seed, traj, t, n))


def gumbel(seed, traj, t, n):
    return np.float32(_load().orc_gumbel(seed, traj, t, n))


def state_before(inst, actions, t):
    """Stock row seen by the order at time t under an action path."""
    lib = _load()
    prod = _c(inst.prod, np.int32)
    act = _c(actions, np.int8)
    x0 = _c(inst.x0, np.int32)
    out = np.empty(inst.N, np.int32)
    rc = lib.orc_state_before(inst.T, inst.N, _p(prod), _p(act), _p(x0), int(t), _p(out))
    if rc != OK:
        raise ValueError("bad t")
    return out


def policy_call(inst, pol, stock_row, k, r, t):
    """One policy decision pi(s, w) for product k, region r, time t."""
    lib = _load()
    args, keep = _args(inst, pol)
    # args layout: T,N,K,R,prod,reg,x0,cost,lam,kind,H,W1,b1,W2,b2,E,seed,traj
    sr = _c(stock_row, np.int32)
    return lib.orc_policy_call(inst.N, inst.R, args[7], args[8], args[9], args[10], *args[11:16],
                               args[16], args[17], _p(sr), int(k), int(r), int(t))
