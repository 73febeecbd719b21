"""B300 Picard-iteration policy simulator for fulfillment optimization.

Thin ctypes binding over the C ABI in ``include/pic.h`` (libpic.so, built in
tree for sm_103a by ``paper_2406_01939_b300.build``).  The functions here only
marshal arguments: every step of the simulation runs in the library's CUDA
kernels.  There is no CPU fallback: if the library or a CUDA device is missing,
calls raise.

Names follow the C ABI: ``pic_create_instance``, ``pic_instance_load``,
``pic_destroy_instance``, ``pic_simulate``, ``pic_create_batch``,
``pic_simulate_batch``, ``pic_policy_grad``, ``pic_simulate_sequential_static``,
``pic_last_error``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpic.so")

PIC_OK, PIC_ERR_INVALID_ARG, PIC_ERR_CUDA, PIC_ERR_OOM = 0, 1, 2, 3
PIC_ERR_NOT_CONVERGED, PIC_ERR_TIMEOUT, PIC_ERR_UNSUPPORTED = 4, 5, 6
PIC_POLICY_GREEDY, PIC_POLICY_DUAL, PIC_POLICY_MLP, PIC_POLICY_GUMBEL = 0, 1, 2, 3
PIC_MODE_PICARD, PIC_MODE_SEQUENTIAL, PIC_MODE_PICARD_PRODUCTS, PIC_MODE_PICARD_ASSIGNED = 0, 1, 2, 3
PIC_MEM_HOST, PIC_MEM_DEVICE = 0, 1
PIC_FLAG_NO_RESET, PIC_FLAG_REUSE_TABLES, PIC_FLAG_TIMING, PIC_FLAG_GROUP_KERNEL = 1, 2, 4, 8
PIC_FLAG_GRAPH, PIC_FLAG_NO_TC, PIC_FLAG_TC, PIC_FLAG_NO_SAT = 16, 32, 64, 128
PIC_FLAG_WARP_GROUP, PIC_FLAG_WAVE, PIC_FLAG_NO_WAVE = 256, 512, 1024

POLICY_KINDS = {"greedy": PIC_POLICY_GREEDY, "dual": PIC_POLICY_DUAL, "mlp": PIC_POLICY_MLP,
                "gumbel": PIC_POLICY_GUMBEL}
MODES = {"picard": PIC_MODE_PICARD, "sequential": PIC_MODE_SEQUENTIAL,
         "products": PIC_MODE_PICARD_PRODUCTS, "assigned": PIC_MODE_PICARD_ASSIGNED}


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pic status {status}: {msg}")
        self.status = status


class pic_instance_desc(C.Structure):
    _fields_ = [("T", C.c_int32), ("N", C.c_int32), ("K", C.c_int32), ("R", C.c_int32),
                ("prod", C.c_void_p), ("reg", C.c_void_p), ("x0", C.c_void_p),
                ("cost", C.c_void_p), ("lam", C.c_void_p), ("mem", C.c_int32),
                ("stream", C.c_void_p), ("cap", C.c_void_p)]


class pic_policy(C.Structure):
    _fields_ = [("kind", C.c_int32), ("hidden", C.c_int32), ("W1", C.c_void_p), ("b1", C.c_void_p),
                ("W2", C.c_void_p), ("b2", C.c_void_p), ("E", C.c_void_p), ("seed", C.c_uint64),
                ("traj", C.c_int32)]


class pic_sim_opts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("num_chunks", C.c_int32), ("max_iters", C.c_int32),
                ("flags", C.c_int32), ("alpha_init", C.c_void_p), ("timeout_ns", C.c_uint64),
                ("out_mem", C.c_int32), ("seg_window", C.c_int32), ("stream", C.c_void_p),
                ("trace", C.c_void_p), ("trace_cap", C.c_int32), ("max_steps", C.c_int32),
                ("proc", C.c_void_p)]


class pic_sim_result(C.Structure):
    _fields_ = [("total_cost", C.c_int64), ("lost", C.c_int64), ("policy_calls", C.c_int64),
                ("iters", C.c_int32), ("num_chunks", C.c_int32), ("rescored", C.c_int64),
                ("seg_replays", C.c_int64), ("launches", C.c_int32), ("prep_ms", C.c_float),
                ("sim_ms", C.c_float), ("total_ms", C.c_float), ("seg_window", C.c_int32),
                ("cta_threads", C.c_int32), ("ctas_per_sm", C.c_int32), ("mlp_calls", C.c_int64),
                ("tc_decisions", C.c_int64), ("sat_decisions", C.c_int64),
                ("near_ties", C.c_int64), ("wave", C.c_int32)]


class pic_traj_result(C.Structure):
    _fields_ = [("total_cost", C.c_int64), ("lost", C.c_int64), ("iters", C.c_int32),
                ("converged", C.c_int32)]


class pic_grad_args(C.Structure):
    _fields_ = [("master", C.c_void_p), ("e_rows", C.c_int32), ("actions", C.c_void_p),
                ("actions_out", C.c_void_p), ("grad", C.c_void_p), ("grad_scale", C.c_double)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libpic.so (raises if it is missing: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing; run paper_2406_01939_b300.build.build()")
            L = C.CDLL(LIB_PATH)
            P = C.c_void_p
            L.pic_create_instance.argtypes = [C.POINTER(pic_instance_desc), C.POINTER(P)]
            L.pic_create_instance.restype = C.c_int
            L.pic_instance_load.argtypes = [P, C.POINTER(pic_instance_desc)]
            L.pic_instance_load.restype = C.c_int
            L.pic_destroy_instance.argtypes = [P]
            L.pic_destroy_instance.restype = None
            L.pic_simulate.argtypes = [P, C.POINTER(pic_policy), C.POINTER(pic_sim_opts), P, P,
                                       C.POINTER(pic_sim_result)]
            L.pic_simulate.restype = C.c_int
            L.pic_create_batch.argtypes = [C.POINTER(pic_instance_desc), C.c_int32, C.POINTER(P)]
            L.pic_create_batch.restype = C.c_int
            L.pic_batch_load.argtypes = [P, C.POINTER(pic_instance_desc), C.c_int32]
            L.pic_batch_load.restype = C.c_int
            L.pic_simulate_batch.argtypes = [P, C.POINTER(pic_policy), C.POINTER(pic_sim_opts), P, P,
                                             C.POINTER(pic_traj_result), C.POINTER(pic_sim_result)]
            L.pic_simulate_batch.restype = C.c_int
            L.pic_policy_grad.argtypes = [P, C.POINTER(pic_policy), C.POINTER(pic_grad_args),
                                          C.POINTER(pic_sim_opts), C.POINTER(C.c_double),
                                          C.POINTER(pic_sim_result)]
            L.pic_policy_grad.restype = C.c_int
            L.pic_simulate_sequential_static.argtypes = [C.POINTER(pic_instance_desc), C.c_int32, P,
                                                         P, C.POINTER(C.c_int64),
                                                         C.POINTER(C.c_int64)]
            L.pic_simulate_sequential_static.restype = C.c_int
            L.pic_last_error.argtypes = []
            L.pic_last_error.restype = C.c_char_p
            _lib = L
    return _lib


def pic_last_error() -> str:
    return lib().pic_last_error().decode()


def _check(status):
    if status != PIC_OK:
        raise PicError(status, pic_last_error())


def _ptr(t):
    """Address of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _stream_handle(stream):
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def make_desc(T, N, K, R, prod, reg, x0, cost, lam=None, mem=PIC_MEM_DEVICE, stream=None,
              cap=None):
    """Build a pic_instance_desc from int32 arrays (torch CUDA tensors for
    mem=PIC_MEM_DEVICE, C-contiguous numpy arrays for PIC_MEM_HOST).  cap: [N]
    node capacity, or None.  The caller keeps the arrays alive for the duration
    of the call."""
    return pic_instance_desc(int(T), int(N), int(K), int(R), _ptr(prod), _ptr(reg), _ptr(x0),
                             _ptr(cost), _ptr(lam), int(mem), _stream_handle(stream), _ptr(cap))


def pic_create_instance(desc: pic_instance_desc) -> int:
    h = C.c_void_p()
    _check(lib().pic_create_instance(C.byref(desc), C.byref(h)))
    return h.value


def pic_instance_load(handle: int, desc: pic_instance_desc) -> None:
    _check(lib().pic_instance_load(C.c_void_p(handle), C.byref(desc)))


def pic_destroy_instance(handle: int) -> None:
    if handle:
        lib().pic_destroy_instance(C.c_void_p(handle))


def make_policy(kind="greedy", W1=None, b1=None, W2=None, b2=None, E=None, hidden=256, seed=0,
                traj=0) -> pic_policy:
    """Policy struct; MLP parameters are device tensors of BF16 bit patterns."""
    k = POLICY_KINDS[kind] if isinstance(kind, str) else int(kind)
    return pic_policy(k, int(hidden), _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2), _ptr(E),
                      int(seed) & 0xFFFFFFFFFFFFFFFF, int(traj))


def make_opts(mode="picard", num_chunks=0, max_iters=0, flags=0, alpha_init=None, timeout_ns=0,
              out_mem=PIC_MEM_DEVICE, seg_window=0, stream=None, trace=None,
              max_steps=0, proc=None) -> pic_sim_opts:
    """trace: optional host int64 numpy array [cap, 6] receiving the per-pass record;
    max_steps: the Picard window (0: none); proc: device int32 [T] process of each
    order (mode "assigned")."""
    if trace is not None and (trace.dtype != np.int64 or trace.ndim != 2 or trace.shape[1] != 6
                              or not trace.flags.c_contiguous):
        raise ValueError("trace must be a C-contiguous int64 array of shape [cap, 6]")
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    return pic_sim_opts(m, int(num_chunks), int(max_iters), int(flags), _ptr(alpha_init),
                        int(timeout_ns), int(out_mem), int(seg_window), _stream_handle(stream),
                        _ptr(trace), 0 if trace is None else int(trace.shape[0]), int(max_steps),
                        _ptr(proc))


def pic_simulate(handle: int, policy: pic_policy, opts: pic_sim_opts, actions_out,
                 final_stock=None, raise_on_error=True):
    """Run one simulation; outputs go to caller-owned buffers (device tensors or
    host numpy arrays per opts.out_mem).  Returns (status, pic_sim_result)."""
    res = pic_sim_result()
    st = lib().pic_simulate(C.c_void_p(handle), C.byref(policy), C.byref(opts), _ptr(actions_out),
                            _ptr(final_stock), C.byref(res))
    if raise_on_error and st != PIC_OK:
        raise PicError(st, pic_last_error())
    return st, res


def pic_create_batch(descs) -> int:
    """Batch instance from a list of pic_instance_desc (all with the same N)."""
    arr = (pic_instance_desc * len(descs))(*descs)
    h = C.c_void_p()
    _check(lib().pic_create_batch(arr, len(descs), C.byref(h)))
    return h.value


def pic_batch_load(handle: int, descs) -> None:
    """Replace every trajectory's inputs of a batch instance (same shapes as at
    creation) with the arrays of a list of pic_instance_desc."""
    arr = (pic_instance_desc * len(descs))(*descs)
    _check(lib().pic_batch_load(C.c_void_p(handle), arr, len(descs)))


def pic_simulate_batch(handle: int, policies, opts: pic_sim_opts, actions_out, final_stock=None,
                       raise_on_error=True):
    """Simulate every trajectory of a batch instance; policies is a list of
    pic_policy (one per trajectory).  Returns (status, pic_sim_result,
    [pic_traj_result])."""
    B = len(policies)
    pols = (pic_policy * B)(*policies)
    traj = (pic_traj_result * B)()
    res = pic_sim_result()
    st = lib().pic_simulate_batch(C.c_void_p(handle), pols, C.byref(opts), _ptr(actions_out),
                                  _ptr(final_stock), traj, C.byref(res))
    if raise_on_error and st != PIC_OK:
        raise PicError(st, pic_last_error())
    return st, res, list(traj)


def pic_policy_grad(handle: int, policies, master, e_rows, opts: pic_sim_opts, actions=None,
                    actions_out=None, grad=None, grad_scale=1.0, raise_on_error=True):
    """REINFORCE objective (and gradient into `grad` if given) of a batch
    instance; master / actions / actions_out / grad are device tensors.  Returns
    (status, objective, pic_sim_result)."""
    B = len(policies)
    pols = (pic_policy * B)(*policies)
    args = pic_grad_args(_ptr(master), int(e_rows), _ptr(actions), _ptr(actions_out), _ptr(grad),
                         float(grad_scale))
    J = C.c_double(0.0)
    res = pic_sim_result()
    st = lib().pic_policy_grad(C.c_void_p(handle), pols, C.byref(args), C.byref(opts), C.byref(J),
                               C.byref(res))
    if raise_on_error and st != PIC_OK:
        raise PicError(st, pic_last_error())
    return st, J.value, res


def pic_simulate_sequential_static(desc: pic_instance_desc, kind, actions_out, final_stock=None,
                                   raise_on_error=True):
    """Sequential simulation with library-owned scratch (no device allocation).
    desc must describe DEVICE arrays; actions_out: CUDA int8 tensor of at least T
    entries; final_stock: None or a CUDA int32 tensor of at least K*N entries.
    Returns (status, total_cost, lost)."""
    import torch
    for name, t, dt, n in (("actions_out", actions_out, torch.int8, desc.T),
                           ("final_stock", final_stock, torch.int32, desc.K * desc.N)):
        if t is None and name == "final_stock":
            continue
        if not (torch.is_tensor(t) and t.is_cuda and t.dtype == dt and t.is_contiguous()
                and t.numel() >= n):
            raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor of at least {n} entries")
    k = POLICY_KINDS[kind] if isinstance(kind, str) else int(kind)
    tc, lost = C.c_int64(0), C.c_int64(0)
    st = lib().pic_simulate_sequential_static(C.byref(desc), k, _ptr(actions_out),
                                              _ptr(final_stock), C.byref(tc), C.byref(lost))
    if raise_on_error and st != PIC_OK:
        raise PicError(st, pic_last_error())
    return st, tc.value, lost.value
