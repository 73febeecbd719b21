"""Python binding of the OWMR inventory-control simulator (include/pic_owmr.h,
Appendix B): argument marshalling only.  Every step of the simulation runs in
libpic.so's CUDA kernels; there is no CPU path."""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np
import torch

from . import PIC_MEM_DEVICE, PIC_MEM_HOST, PIC_MODE_PICARD, PIC_MODE_SEQUENTIAL, PIC_OK, \
    PIC_FLAG_TIMING, PicError, _ptr, _stream_handle, lib, pic_last_error

__all__ = ["DeviceOwmr", "DeviceOwmrNet", "pic_owmr_create", "pic_owmr_simulate",
           "pic_owmr_destroy", "pic_owmr_desc", "pic_owmr_policy", "pic_owmr_opts",
           "pic_owmr_result", "PIC_MEM_HOST"]

P_ = C.c_void_p

class pic_owmr_desc(C.Structure):
    _fields_ = [("T", C.c_int32), ("N", C.c_int32), ("ret", P_), ("dem", P_), ("ex", P_), ("cap", P_),
                ("x0r", P_), ("sl", P_), ("Sl", P_), ("X0", C.c_int32), ("s", C.c_int32),
                ("S", C.c_int32), ("mem", C.c_int32), ("stream", P_)]


class pic_owmr_policy(C.Structure):
    _fields_ = [("hidden", C.c_int32), ("W1", P_), ("b1", P_), ("W2", P_), ("b2", P_),
                ("w3", P_), ("b3", P_)]


class pic_owmr_opts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("num_procs", C.c_int32), ("max_iters", C.c_int32),
                ("flags", C.c_int32), ("alpha_init", P_), ("timeout_ns", C.c_int64),
                ("max_steps", C.c_int32)]


class pic_owmr_result(C.Structure):
    _fields_ = [("iters", C.c_int32), ("procs", C.c_int32), ("replenishments", C.c_int64),
                ("lost", C.c_int64), ("shipped", C.c_int64), ("policy_calls", C.c_int64),
                ("eval_rounds", C.c_int64), ("launches", C.c_int32), ("ms_total", C.c_float),
                ("near_ties", C.c_int64)]


_bound = False


def _lib():
    global _bound
    L = lib()
    if not _bound:
        L.pic_owmr_create.argtypes = [C.POINTER(pic_owmr_desc), C.POINTER(P_)]
        L.pic_owmr_create.restype = C.c_int
        L.pic_owmr_simulate.argtypes = [P_, C.POINTER(pic_owmr_policy), C.POINTER(pic_owmr_opts),
                                        P_, P_, C.c_int32, C.POINTER(pic_owmr_result), P_]
        L.pic_owmr_simulate.restype = C.c_int
        L.pic_owmr_destroy.argtypes = [P_]
        L.pic_owmr_destroy.restype = None
        _bound = True
    return L


def _check(status):
    if status != PIC_OK:
        raise PicError(status, pic_last_error())


def pic_owmr_create(desc: pic_owmr_desc) -> int:
    h = P_()
    _check(_lib().pic_owmr_create(C.byref(desc), C.byref(h)))
    return h.value


def pic_owmr_simulate(handle, policy, opts, actions_out, state_out=None, out_mem=PIC_MEM_DEVICE,
                      stream=None):
    res = pic_owmr_result()
    st = _lib().pic_owmr_simulate(handle, C.byref(policy), C.byref(opts), _ptr(actions_out),
                                  _ptr(state_out), int(out_mem), C.byref(res),
                                  _stream_handle(stream))
    return st, res


def pic_owmr_destroy(handle) -> None:
    _lib().pic_owmr_destroy(handle)


def _dev_i32(a, device):
    return torch.from_numpy(np.array(a, dtype=np.int32, copy=True)).to(device)


def _dev_u16(a, device):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).to(device)


class DeviceOwmrNet:
    """The retailer network's BF16 parameters on the device."""

    def __init__(self, net, device="cuda"):
        self.H = int(net.H)
        self.t = [_dev_u16(getattr(net, k), device) for k in ("W1", "b1", "W2", "b2", "w3", "b3")]

    def policy(self) -> pic_owmr_policy:
        return pic_owmr_policy(self.H, *[_ptr(x) for x in self.t])


class DeviceOwmr:
    """An OWMR instance resident on the device (pic_owmr_create from device
    arrays)."""

    def __init__(self, inst, device="cuda", stream=None):
        self.inst = inst
        self.device = torch.device(device)
        self.T, self.N = int(inst.T), int(inst.N)
        arrs = [inst.ret, inst.dem, inst.ex, inst.cap, inst.x0r, inst.sl, inst.Sl]
        self._keep = [_dev_i32(a, self.device) for a in arrs]
        d = pic_owmr_desc(self.T, self.N, *[_ptr(x) for x in self._keep], int(inst.X0),
                          int(inst.s), int(inst.S), PIC_MEM_DEVICE, _stream_handle(stream))
        self.handle = pic_owmr_create(d)

    def close(self):
        if self.handle:
            pic_owmr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def simulate(self, net=None, mode="picard", num_procs=0, max_iters=0, alpha_init=None,
                 timing=False, timeout_ns=0, raise_on_error=True, stream=None, max_steps=0,
                 flags=0):
        """Run the Picard iteration (or the sequential baseline) under the
        retailer rule, with the network `net` (a DeviceOwmrNet, an OwmrNet, or
        None).  Returns device tensors and the call's statistics."""
        if net is not None and not isinstance(net, DeviceOwmrNet):
            net = DeviceOwmrNet(net, self.device)
        pol = net.policy() if net is not None else pic_owmr_policy(0)
        init = None
        if alpha_init is not None:
            init = alpha_init if torch.is_tensor(alpha_init) else _dev_i32(alpha_init, self.device)
        opts = pic_owmr_opts(PIC_MODE_PICARD if mode == "picard" else PIC_MODE_SEQUENTIAL,
                             int(num_procs), int(max_iters),
                             (PIC_FLAG_TIMING if timing else 0) | int(flags),
                             _ptr(init), int(timeout_ns), int(max_steps))
        act = torch.empty(max(self.T, 1), dtype=torch.int32, device=self.device)
        state = torch.empty(self.N + 1, dtype=torch.int32, device=self.device)
        st, res = pic_owmr_simulate(self.handle, pol, opts, act, state, PIC_MEM_DEVICE, stream)
        if st != PIC_OK and raise_on_error:
            raise PicError(st, pic_last_error())
        act = act[:self.T]
        return {"status": st, "actions": act, "q": act >> 1, "r": act & 1, "state": state,
                "iters": res.iters, "procs": res.procs, "R": res.replenishments,
                "lost": res.lost, "shipped": res.shipped, "policy_calls": res.policy_calls,
                "eval_rounds": res.eval_rounds, "near_ties": res.near_ties, "launches": res.launches, "ms": res.ms_total,
                "_keep": (net, init)}
