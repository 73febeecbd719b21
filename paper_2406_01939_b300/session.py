"""Marshalling helpers over the C ABI: put an instance's arrays into device
memory with torch, hold the instance handle, and call ``pic_simulate`` with
device output buffers.  No simulation arithmetic happens here."""
from __future__ import annotations

import numpy as np
import torch

from . import (PIC_MEM_DEVICE, PIC_MEM_HOST, make_desc, make_opts, make_policy, pic_batch_load,
               pic_create_batch, pic_create_instance, pic_destroy_instance, pic_instance_load, pic_simulate,
               pic_simulate_batch)


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
        cap = getattr(inst, "cap", None)
        d["cap"] = None if cap is None else _dev(cap.astype(np.int32), self.device)
        return d

    def _desc(self, arrs, stream, mem=PIC_MEM_DEVICE):
        i = self.inst
        return make_desc(i.T, i.N, i.K, i.R, arrs["prod"], arrs["reg"], arrs["x0"], arrs["cost"],
                         arrs["lam"], mem=mem, stream=stream, cap=arrs.get("cap"))

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
                 trace=None, max_steps=0, proc=None):
        i = self.inst
        dp = policy if isinstance(policy, DevicePolicy) else DevicePolicy(policy, self.device)
        act = out if out is not None else torch.empty(i.T, dtype=torch.int8, device=self.device)
        stock = torch.empty((i.K, i.N), dtype=torch.int32, device=self.device) if want_stock else None
        ai = None
        if alpha_init is not None:
            ai = torch.as_tensor(np.ascontiguousarray(alpha_init, dtype=np.int8)).to(self.device) \
                if not torch.is_tensor(alpha_init) else alpha_init
        pr = None
        if proc is not None:
            pr = proc if torch.is_tensor(proc) else \
                torch.as_tensor(np.ascontiguousarray(proc, dtype=np.int32)).to(self.device)
        opts = make_opts(mode, num_chunks, max_iters, flags, ai, timeout_ns, PIC_MEM_DEVICE,
                         seg_window, self.stream, trace, max_steps, pr)
        st, res = pic_simulate(self.handle, dp.struct, opts, act, stock, raise_on_error)
        return {"status": st, "actions": act, "final_stock": stock, "total_cost": res.total_cost,
                "lost": res.lost, "iters": res.iters, "policy_calls": res.policy_calls,
                "num_chunks": res.num_chunks, "rescored": res.rescored,
                "seg_replays": res.seg_replays, "launches": res.launches, "prep_ms": res.prep_ms,
                "sim_ms": res.sim_ms, "total_ms": res.total_ms, "seg_window": res.seg_window,
                "cta_threads": res.cta_threads, "ctas_per_sm": res.ctas_per_sm,
                "mlp_calls": res.mlp_calls, "tc_decisions": res.tc_decisions,
                "sat_decisions": res.sat_decisions, "near_ties": res.near_ties, "wave": bool(res.wave)}

    def close(self):
        if self.handle:
            pic_destroy_instance(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceBatch:
    """A batch of trajectories (list of synth.Instance, same N) as one library
    batch instance.  Outputs of ``simulate`` are concatenated in trajectory
    order; ``offsets`` gives each trajectory's first order."""

    def __init__(self, insts, device="cuda", stream=None, mem=PIC_MEM_DEVICE):
        self.insts = list(insts)
        self.device = device
        self.stream = stream
        self.T = int(sum(i.T for i in self.insts))
        self.K = int(sum(i.K for i in self.insts))
        self.N = int(self.insts[0].N)
        self.offsets = np.concatenate([[0], np.cumsum([i.T for i in self.insts])]).astype(np.int64)
        self.koffsets = np.concatenate([[0], np.cumsum([i.K for i in self.insts])]).astype(np.int64)
        keep, descs = self._descs(self.insts, mem)
        self.handle = pic_create_batch(descs)
        del keep  # the batch holds its own device copies

    def _descs(self, insts, mem):
        """Descriptors of insts' arrays (device copies for PIC_MEM_DEVICE, the
        host arrays themselves for PIC_MEM_HOST) and the arrays to keep alive."""
        device, stream = self.device, self.stream
        keep, descs = [], []
        for i in insts:
            if mem == PIC_MEM_DEVICE:
                a = {k: _dev(getattr(i, k).astype(np.int32), device) for k in ("prod", "reg", "x0", "cost")}
                a["lam"] = None if i.lam is None else _dev(i.lam.astype(np.int32), device)
            else:
                a = {k: np.ascontiguousarray(getattr(i, k), dtype=np.int32)
                     for k in ("prod", "reg", "x0", "cost")}
                a["lam"] = None if i.lam is None else np.ascontiguousarray(i.lam, dtype=np.int32)
            cap = getattr(i, "cap", None)  # not supported in a batch: the library rejects it
            if cap is not None:
                a["cap"] = (_dev(cap.astype(np.int32), device) if mem == PIC_MEM_DEVICE
                            else np.ascontiguousarray(cap, dtype=np.int32))
            keep.append(a)
            descs.append(make_desc(i.T, i.N, i.K, i.R, a["prod"], a["reg"], a["x0"], a["cost"],
                                   a["lam"], mem=mem, stream=stream, cap=a.get("cap")))
        return keep, descs

    def load(self, insts, mem=PIC_MEM_DEVICE):
        """Replace every trajectory's inputs with those of insts (the same shapes,
        lam present where it was), reusing the batch's device memory
        (pic_batch_load); PIC_MEM_HOST copies C-contiguous host arrays."""
        insts = list(insts)
        keep, descs = self._descs(insts, mem)
        pic_batch_load(self.handle, descs)
        del keep
        self.insts = insts

    def simulate(self, policies, mode="picard", num_chunks=0, max_iters=0, flags=0, alpha_init=None,
                 timeout_ns=0, seg_window=0, want_stock=True, raise_on_error=True, out=None,
                 trace=None, out_mem=PIC_MEM_DEVICE, max_steps=0):
        """policies: list of synth.Policy or DevicePolicy, one per trajectory (MLP
        kinds must share one parameter set: pass the same DevicePolicy object or
        Policies holding the same MLPParams object)."""
        dps, cache = [], {}
        for p in policies:
            if isinstance(p, DevicePolicy):
                dps.append(p)
                continue
            key = id(p.mlp) if p.mlp is not None else None
            if key is not None and key in cache:
                base = cache[key]
            else:
                base = DevicePolicy(p, self.device)
                if key is not None:
                    cache[key] = base
            dp = DevicePolicy.__new__(DevicePolicy)
            dp.kind, dp.tensors, dp.hidden = p.kind, base.tensors, base.hidden
            dp.struct = make_policy(p.kind, hidden=dp.hidden, seed=p.seed, traj=p.traj, **dp.tensors)
            dps.append(dp)
        host = out_mem == PIC_MEM_HOST
        if out is not None:
            act = out
        elif host:
            act = np.empty(self.T, np.int8)
        else:
            act = torch.empty(self.T, dtype=torch.int8, device=self.device)
        stock = None
        if want_stock:
            stock = (np.empty((self.K, self.N), np.int32) if host else
                     torch.empty((self.K, self.N), dtype=torch.int32, device=self.device))
        ai = None
        if alpha_init is not None:
            ai = alpha_init if torch.is_tensor(alpha_init) else \
                torch.as_tensor(np.ascontiguousarray(alpha_init, dtype=np.int8)).to(self.device)
        opts = make_opts(mode, num_chunks, max_iters, flags, ai, timeout_ns, out_mem, seg_window,
                         self.stream, trace, max_steps)
        st, res, traj = pic_simulate_batch(self.handle, [d.struct for d in dps], opts, act, stock,
                                           raise_on_error)
        return {"status": st, "actions": act, "final_stock": stock, "total_cost": res.total_cost,
                "lost": res.lost, "iters": res.iters, "policy_calls": res.policy_calls,
                "num_chunks": res.num_chunks, "seg_window": res.seg_window,
                "cta_threads": res.cta_threads, "ctas_per_sm": res.ctas_per_sm,
                "mlp_calls": res.mlp_calls, "tc_decisions": res.tc_decisions,
                "sat_decisions": res.sat_decisions, "near_ties": res.near_ties, "wave": bool(res.wave),
                "rescored": res.rescored, "seg_replays": res.seg_replays,
                "launches": res.launches, "prep_ms": res.prep_ms,
                "sim_ms": res.sim_ms, "total_ms": res.total_ms,
                "traj": [{"total_cost": t.total_cost, "lost": t.lost, "iters": t.iters,
                          "converged": t.converged} for t in traj]}

    def split(self, arr):
        """Per-trajectory views of a concatenated action array."""
        return [arr[self.offsets[b]:self.offsets[b + 1]] for b in range(len(self.insts))]

    def split_stock(self, arr):
        return [arr[self.koffsets[b]:self.koffsets[b + 1]] for b in range(len(self.insts))]

    def close(self):
        if self.handle:
            pic_destroy_instance(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
