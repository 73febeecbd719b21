"""pic_simulate_sequential_static: the sequential simulator for callers that may
not allocate device memory (its scratch is a fixed array owned by the library).
Checked through the C ABI against the allocating entry point (pic_simulate in
sequential mode) on two calls in a row; integer outputs must be identical.
This file is collected last so that a stop-at-first-failure run has already run
every other test."""
import numpy as np
import pytest
import torch

import paper_2406_01939_b300 as pic
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.session import DeviceInstance
from paper_2406_01939_b300.synth import Policy

pytestmark = pytest.mark.gpu


def _device_desc(inst, dev="cuda"):
    arrs = {k: torch.from_numpy(np.ascontiguousarray(getattr(inst, k), np.int32)).to(dev)
            for k in ("prod", "reg", "x0", "cost")}
    arrs["lam"] = None if inst.lam is None else torch.from_numpy(
        np.ascontiguousarray(inst.lam, np.int32)).to(dev)
    desc = pic.make_desc(inst.T, inst.N, inst.K, inst.R, arrs["prod"], arrs["reg"], arrs["x0"],
                         arrs["cost"], arrs["lam"], mem=pic.PIC_MEM_DEVICE)
    return desc, arrs


def test_static_scratch_matches_allocating_entry_point_twice():
    cases = [(synth.dual_large(0, T=1 << 16, K=2000, R=200), "dual"),
             (synth.greedy_small(3), "greedy")]
    for inst, kind in cases:  # two calls in a row share the library's scratch array
        desc, arrs = _device_desc(inst)
        act = torch.empty(inst.T, dtype=torch.int8, device="cuda")
        stock = torch.empty((inst.K, inst.N), dtype=torch.int32, device="cuda")
        st, tc, lost = pic.pic_simulate_sequential_static(desc, kind, act, stock)
        assert st == pic.PIC_OK
        ref = DeviceInstance(inst).simulate(Policy(kind), "sequential")
        assert torch.equal(act, ref["actions"])
        assert torch.equal(stock, ref["final_stock"])
        assert tc == ref["total_cost"] and lost == ref["lost"]


def test_static_scratch_rejects_oversized_instances():
    inst = synth.make_instance(100, 64, 20_000, 4, seed=1, stock="uniform")  # K*N > limit
    desc, arrs = _device_desc(inst)
    act = torch.empty(inst.T, dtype=torch.int8, device="cuda")
    st, _, _ = pic.pic_simulate_sequential_static(desc, "greedy", act, raise_on_error=False)
    assert st == pic.PIC_ERR_INVALID_ARG
    assert "static scratch limit" in pic.pic_last_error()
