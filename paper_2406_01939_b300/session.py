"""Marshalling helpers over the C ABI: put an instance's arrays into device
memory with torch, hold the instance handle, and call ``pic_simulate`` with
device output buffers.  No simulation arithmetic happens here."""
from __future__ import annotations

import numpy as np
import torch

from . import (PIC_MEM_DEVICE, PIC_MEM_HOST, make_desc, make_opts, make_policy, pic_create_instance,
               pic_destroy_instance, pic_instance_load, pic_simulate)


def _dev(a, device):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


def bf16_bits_to_device(a, device):
    """uint16 BF16 bit patterns -> int16 device tensor (same bits)."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).to(device)


class DevicePolicy:
    """A synth.Policy with its MLP parameters resident on the device."""

    def __init__(self, pol, device="cuda"):
        self.kind = pol.kind
        self.tensors = {}
        if pol.mlp is not None:
            for k in ("W1", "b1", "W2", "b2", "E"):
                self.tensors[k] = bf16_bits_to_device(getattr(pol.mlp, k), device)
            self.hidden = pol.mlp.H
        else:
            self.hidden = 256
        self.struct = make_policy(pol.kind, hidden=self.hidden, seed=pol.seed, traj=pol.traj,
                                  **self.tensors)


class DeviceInstance:
    """One trajectory's inputs in device memory plus its library handle."""

    def __init__(self, inst, device="cuda", stream=None):
        self.inst = inst
        self.device = device
        self.stream = stream
        self.arrays = self._upload(inst)
        self.handle = pic_create_instance(self._desc(self.arrays, stream))

    def _upload(self, inst):
        d = {k: _dev(getattr(inst, k).astype(np.int32), self.device)
             for k in ("prod", "reg", "x0", "cost")}
        d["lam"] = None if inst.lam is None else _dev(inst.lam.astype(np.int32), self.device)
        return d

    def _desc(self, arrs, stream, mem=PIC_MEM_DEVICE):
        i = self.inst
        return make_desc(i.T, i.N, i.K, i.R, arrs["prod"], arrs["reg"], arrs["x0"], arrs["cost"],
                         arrs["lam"], mem=mem, stream=stream)

    def load(self, inst):
        """Stream new inputs of the same shape into this instance."""
        self.inst = inst
        self.arrays = self._upload(inst)
        pic_instance_load(self.handle, self._desc(self.arrays, self.stream))

    def load_host(self, host_arrays):
        """Load from host numpy arrays (the library copies them to the device)."""
        pic_instance_load(self.handle, self._desc(host_arrays, self.stream, mem=PIC_MEM_HOST))

    def simulate(self, policy, mode="picard", num_chunks=0, max_iters=0, flags=0, alpha_init=None,
                 timeout_ns=0, seg_window=0, want_stock=True, raise_on_error=True, out=None,
                 trace=None):
        i = self.inst
        dp = policy if isinstance(policy, DevicePolicy) else DevicePolicy(policy, self.device)
        act = out if out is not None else torch.empty(i.T, dtype=torch.int8, device=self.device)
        stock = torch.empty((i.K, i.N), dtype=torch.int32, device=self.device) if want_stock else None
        ai = None
        if alpha_init is not None:
            ai = torch.as_tensor(np.ascontiguousarray(alpha_init, dtype=np.int8)).to(self.device) \
                if not torch.is_tensor(alpha_init) else alpha_init
        opts = make_opts(mode, num_chunks, max_iters, flags, ai, timeout_ns, PIC_MEM_DEVICE,
                         seg_window, self.stream, trace)
        st, res = pic_simulate(self.handle, dp.struct, opts, act, stock, raise_on_error)
        return {"status": st, "actions": act, "final_stock": stock, "total_cost": res.total_cost,
                "lost": res.lost, "iters": res.iters, "policy_calls": res.policy_calls,
                "num_chunks": res.num_chunks, "rescored": res.rescored,
                "seg_replays": res.seg_replays, "launches": res.launches, "prep_ms": res.prep_ms,
                "sim_ms": res.sim_ms, "total_ms": res.total_ms}

    def close(self):
        if self.handle:
            pic_destroy_instance(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
