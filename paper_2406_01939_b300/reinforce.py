"""REINFORCE objective of the MLP fulfilment policy as a torch.autograd.Function.

Forward simulates the batch's trajectories under the policy whose parameters
are BF16(master) and evaluates J = sum_t log pi(a_t | s_t) G_t in the library's
kernels (``pic_policy_grad`` without a gradient buffer); backward runs the
library's hand-written gradient kernel along the same paths.  This module only
marshals arguments: the flat parameter layout of the C ABI is
W1 [(2N+16), 256] | b1 [256] | W2 [256, N] | b2 [N] | E [e_rows, 16].
"""
from __future__ import annotations

import numpy as np
import torch

from . import make_opts, make_policy, pic_policy_grad
from .synth import bf16_to_f32


def param_shapes(N, e_rows, H=256):
    return {"W1": (2 * N + 16, H), "b1": (H,), "W2": (H, N), "b2": (N,), "E": (e_rows, 16)}


def flat_from_mlp(mlp, device="cuda"):
    """FP32 master vector holding an MLPParams' BF16 values exactly."""
    parts = [bf16_to_f32(getattr(mlp, k)).ravel() for k in ("W1", "b1", "W2", "b2", "E")]
    return torch.from_numpy(np.concatenate(parts).astype(np.float32)).to(device)


def split_flat(v, N, e_rows):
    """Views of a flat parameter (or gradient) vector by name."""
    out, o = {}, 0
    for k, shp in param_shapes(N, e_rows).items():
        n = int(np.prod(shp))
        out[k] = v[o:o + n].view(*shp)
        o += n
    return out


class Reinforce:
    """Policy-gradient objective over a DeviceBatch.  kinds: 'mlp' or 'gumbel'
    per trajectory; seeds / trajs key the Gumbel noise."""

    def __init__(self, batch, kinds, seeds, trajs, e_rows, num_chunks=0, seg_window=0, stream=None,
                 flags=0):
        self.batch = batch
        self.e_rows = int(e_rows)
        self.pols = [make_policy(k, hidden=256, seed=int(s), traj=int(t))
                     for k, s, t in zip(kinds, seeds, trajs)]
        self.opts = make_opts("picard", num_chunks, seg_window=seg_window, stream=stream, flags=flags)
        self.last_actions = None
        self.last_result = None

    def objective(self, master, actions=None, actions_out=None):
        _, J, res = pic_policy_grad(self.batch.handle, self.pols, master, self.e_rows, self.opts,
                                    actions=actions, actions_out=actions_out)
        return J, res

    def step(self, master, grad, actions_out=None):
        """One policy-gradient step in one call: simulate the paths under
        BF16(master), then J and dJ/dtheta along them.  Returns (J, result)."""
        _, J, res = pic_policy_grad(self.batch.handle, self.pols, master, self.e_rows, self.opts,
                                    actions_out=actions_out, grad=grad)
        return J, res

    def gradient(self, master, actions, grad, scale=1.0):
        _, J, _ = pic_policy_grad(self.batch.handle, self.pols, master, self.e_rows, self.opts,
                                  actions=actions, grad=grad, grad_scale=scale)
        return J

    def __call__(self, master):
        return _ReinforceFn.apply(master, self)


class _ReinforceFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, master, rf):
        acts = torch.empty(rf.batch.T, dtype=torch.int8, device=master.device)
        J, res = rf.objective(master, actions_out=acts)
        rf.last_actions, rf.last_result = acts, res
        ctx.rf = rf
        ctx.save_for_backward(master, acts)
        return torch.tensor(J, dtype=torch.float64, device=master.device)

    @staticmethod
    def backward(ctx, gJ):
        master, acts = ctx.saved_tensors
        g = torch.empty_like(master)
        ctx.rf.gradient(master, acts, g, scale=float(gJ))
        return g, None
