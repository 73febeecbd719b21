"""CPU oracle for the OWMR inventory-control extension (Appendix B) -- TEST
INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU legs may import it.  The arithmetic lives in ``owmr_oracle.c``
(plain C, ``-ffp-contract=off``); this module only marshals arguments.

Inputs are duck-typed: an instance needs T, N, ret, dem, ex, cap, x0r, sl, Sl
(int arrays), X0, s, S (ints); a network needs H and W1 [3][H], b1 [H],
W2 [H][H] (input-major), b2 [H], w3 [H], b3 [1] as BF16 bit patterns (uint16),
or is None.

Parity status: every function is pinned in ``tests/test_oracle_owmr.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "owmr_oracle.c")
_LIB = os.path.join(_HERE, "libowmr_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NOT_CONVERGED = 0, 1, 4


def build(force: bool = False) -> str:
    """Compile owmr_oracle.c with gcc (IEEE FP32, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P, i32 = C.c_void_p, C.c_int32
            model = [i32, i32, P, P, P, P, P, P, P, i32, i32, i32, i32, P, P, P, P, P, P]
            lib.orc_owmr_seq.argtypes = model + [P, P, P]
            lib.orc_owmr_seq.restype = C.c_int
            lib.orc_owmr_picard_literal.argtypes = model + [i32, P, i32, i32, P, P, P, P, P]
            lib.orc_owmr_picard_literal.restype = C.c_int
            lib.orc_owmr_picard_walk.argtypes = model + [i32, P, i32, i32, P, P, P, P, P, P, P]
            lib.orc_owmr_picard_walk.restype = C.c_int
            lib.owmr_mlp.argtypes = [P, i32, i32, i32, P, P]
            lib.owmr_mlp.restype = C.c_float
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _u16(a):
    return np.ascontiguousarray(a, dtype=np.uint16)


def _model(inst, net):
    keep = [_i32(inst.ret), _i32(inst.dem), _i32(inst.ex), _i32(inst.cap), _i32(inst.x0r),
            _i32(inst.sl), _i32(inst.Sl)]
    if net is None:
        nk, H = [None] * 6, 0
    else:
        nk = [_u16(net.W1), _u16(net.b1), _u16(net.W2), _u16(net.b2), _u16(net.w3),
              _u16(net.b3)]
        H = int(net.H)
    keep += nk
    args = [int(inst.T), int(inst.N)] + [_p(a) for a in keep[:7]] + \
        [int(inst.X0), int(inst.s), int(inst.S), H] + [_p(a) for a in nk]
    return args, keep


def _err(rc, what):
    if rc == ERR_ARG:
        raise ValueError(f"{what}: invalid arguments")


def seq_sim(inst, net=None):
    """Sequential simulation of the OWMR model (Appendix B.1 dynamics, B.2
    policy).  Returns actions (2 q + r per step), q, r, x_final (x0 first),
    R (replenishments), lost, shipped and evals (network calls).

    Pins: a hand-derived trace; conservation (retailer stock change = shipped
    - sold); central inventory between replenishments = S - units shipped;
    with no retailer orders, no replenishment; special cases."""
    lib = _load()
    args, keep = _model(inst, net)
    T, N = int(inst.T), int(inst.N)
    act = np.zeros(max(T, 1), np.int32)
    xf = np.zeros(N + 1, np.int32)
    st = np.zeros(4, np.int64)
    rc = lib.orc_owmr_seq(*args, _p(act), _p(xf), _p(st))
    _err(rc, "owmr seq_sim")
    act = act[:T]
    return {"actions": act, "q": act >> 1, "r": act & 1, "x_final": xf, "R": int(st[0]),
            "lost": int(st[1]), "shipped": int(st[2]), "evals": int(st[3])}


def _procs(inst, proc):
    proc = _i32(proc)
    P = int(proc.max()) + 1 if proc.size else 1
    return proc, P


def _run_picard(fn, inst, net, proc, max_iters, alpha_init, record, extra, window=0):
    lib = _load()
    args, keep = _model(inst, net)
    proc, P = _procs(inst, proc)
    T = int(inst.T)
    if max_iters is None:
        max_iters = 2 * T + 2 + (2 * (T // window + 1) if window else 0)
    init = None if alpha_init is None else _i32(alpha_init)
    act = np.zeros(max(T, 1), np.int32)
    iters = np.zeros(1, np.int32)
    ev = np.zeros(1, np.int64)
    rec = np.zeros((max_iters, max(T, 1)), np.int32) if record else None
    rc = getattr(lib, fn)(*args, P, _p(proc), int(max_iters), int(window), _p(init), _p(act),
                          _p(iters),
                          _p(rec), _p(ev), *[_p(a) for a in extra])
    _err(rc, fn)
    k = int(iters[0])
    out = {"actions": act[:T], "iters": k, "converged": rc == OK, "evals": int(ev[0])}
    if record:
        out["iterates"] = rec[:k, :T]
    return out


def picard_literal(inst, net, proc, max_iters=None, alpha_init=None, record=False, window=0):
    """Algorithm 1 with the retailer partition (processor of retailer n =
    proc[n]), every processor replaying the whole horizon each pass.

    Pins: Prop. 1 (fixed point = sequential path; the first step that differs
    from it moves strictly forward every pass); one processor = one pass plus a
    confirming pass;
    Theorem B.1: with s >= every retailer capacity and x0 > s, alpha^k equals
    the sequential path for every k >= 2R + 1 (R replenishments of the
    sequential path), and for k >= 1 when R = 0.

    window > 0: the max_steps window of Appendix A.3 in steps (see
    owmr_oracle.c).  Pins: fixed point = sequential path for every window; a
    window >= T gives the unwindowed iterates; one processor on a path whose
    every action is nonzero takes exactly 2 ceil(T / window) passes."""
    return _run_picard("orc_owmr_picard_literal", inst, net, proc, max_iters, alpha_init,
                       record, [], window)


def picard_walk(inst, net, proc, max_iters=None, alpha_init=None, record=False, window=0):
    """The same iteration through prefix quantities of the cache and a walk of
    each processor's own steps (the organisation the GPU path uses), with
    memoised policy calls.  Pins: every iterate equal to picard_literal's."""
    T, N = int(inst.T), int(inst.N)
    xf = np.zeros(N + 1, np.int32)
    st = np.zeros(4, np.int64)
    out = _run_picard("orc_owmr_picard_walk", inst, net, proc, max_iters, alpha_init, record,
                      [xf, st], window)
    out.update(x_final=xf, R=int(st[0]), lost=int(st[1]), shipped=int(st[2]))
    return out


class _Net(C.Structure):
    _fields_ = [("H", C.c_int), ("W1", C.c_void_p), ("b1", C.c_void_p), ("W2", C.c_void_p),
                ("b2", C.c_void_p), ("w3", C.c_void_p), ("b3", C.c_void_p)]


def mlp(net, y, d, e=0):
    """The network's FP32 output z for features (y, d, e / 4096) in the fixed
    order of owmr_mlp().  Pin: within the FP32 rounding bound of an FP64
    evaluation."""
    lib = _load()
    keep = [_u16(net.W1), _u16(net.b1), _u16(net.W2), _u16(net.b2), _u16(net.w3), _u16(net.b3)]
    s = _Net(int(net.H), *[_p(a) for a in keep])
    h1 = np.zeros(int(net.H), np.float32)
    h2 = np.zeros(int(net.H), np.float32)
    return float(lib.owmr_mlp(C.byref(s), int(y), int(d), int(e), _p(h1), _p(h2)))
