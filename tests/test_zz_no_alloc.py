"""pic_simulate_sequential_static: the sequential simulator for callers that may
not allocate device memory (its scratch is a fixed array owned by the library).
Checked through the C ABI against the allocating entry point (pic_simulate in
sequential mode) on two calls in a row, and against the CPU oracle's sequential
simulation; integer outputs must be identical.  This file is collected last so
that a stop-at-first-failure run has already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
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


CASES = [(lambda: synth.dual_large(0, T=1 << 16, K=2000, R=200), "dual"),   # N = 64
         (lambda: synth.greedy_small(3), "greedy"),                          # N = 8
         (lambda: synth.make_instance(5000, 100, 40, 30, seed=7, stock="poisson",
                                      with_lam=True), "dual"),              # N = 100
         (lambda: synth.greedy_small(4, T=0), "greedy")]                     # T = 0


def test_static_scratch_matches_allocating_entry_point_twice():
    for make, kind in CASES:
        inst = make()
        desc, arrs = _device_desc(inst)
        want = oracle.seq_sim(inst, Policy(kind))
        ref = DeviceInstance(inst).simulate(Policy(kind), "sequential")
        for _ in range(2):  # two calls in a row share the library's scratch array
            act = torch.full((max(inst.T, 1),), 99, dtype=torch.int8, device="cuda")
            stock = torch.empty((inst.K, inst.N), dtype=torch.int32, device="cuda")
            st, tc, lost = pic.pic_simulate_sequential_static(desc, kind, act, stock)
            assert st == pic.PIC_OK
            if inst.T:
                assert torch.equal(act[:inst.T], ref["actions"])
                np.testing.assert_array_equal(act[:inst.T].cpu().numpy(), want["actions"])
            assert torch.equal(stock, ref["final_stock"])
            np.testing.assert_array_equal(stock.cpu().numpy(), want["x_final"])
            assert tc == ref["total_cost"] == want["total_cost"]
            assert lost == ref["lost"] == want["lost"]


def test_static_call_takes_no_device_memory():
    """After a first call (which resolves the scratch array's address), further
    calls leave the device's free memory unchanged."""
    inst = synth.dual_large(1, T=1 << 15, K=1000, R=100)
    desc, arrs = _device_desc(inst)
    act = torch.empty(inst.T, dtype=torch.int8, device="cuda")
    stock = torch.empty((inst.K, inst.N), dtype=torch.int32, device="cuda")
    pic.pic_simulate_sequential_static(desc, "dual", act, stock)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        pic.pic_simulate_sequential_static(desc, "dual", act, stock)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_scratch_rejects_oversized_instances():
    inst = synth.make_instance(100, 64, 20_000, 4, seed=1, stock="uniform")  # K*N > limit
    desc, arrs = _device_desc(inst)
    act = torch.empty(inst.T, dtype=torch.int8, device="cuda")
    st, _, _ = pic.pic_simulate_sequential_static(desc, "greedy", act, raise_on_error=False)
    assert st == pic.PIC_ERR_INVALID_ARG
    assert "static scratch limit" in pic.pic_last_error()


def test_static_scratch_rejects_host_and_short_arrays():
    """The C entry point checks every pointer on the host before any launch: a
    host array, or a device array shorter than the call writes, is INVALID_ARG."""
    inst = synth.greedy_small(5)
    desc, arrs = _device_desc(inst)
    L = pic.lib()
    tc, lost = C.c_int64(0), C.c_int64(0)
    host_act = np.empty(inst.T, np.int8)
    st = L.pic_simulate_sequential_static(C.byref(desc), pic.POLICY_KINDS["greedy"],
                                          C.c_void_p(host_act.ctypes.data), None,
                                          C.byref(tc), C.byref(lost))
    assert st == pic.PIC_ERR_INVALID_ARG and "actions_out" in pic.pic_last_error()
    act = torch.empty(inst.T, dtype=torch.int8, device="cuda")
    # a buffer whose last 16 bytes are handed over as final_stock (K*N int32 =
    # 512 bytes would run past the end of its allocation); the test allocates it
    # itself (2 MiB, a whole allocation granule) so that its extent is exact
    rt = C.CDLL("libcudart.so.13")
    buf = C.c_void_p()
    size = 2 << 20
    assert rt.cudaMalloc(C.byref(buf), C.c_size_t(size)) == 0
    try:
        st = L.pic_simulate_sequential_static(C.byref(desc), pic.POLICY_KINDS["greedy"],
                                              C.c_void_p(act.data_ptr()),
                                              C.c_void_p(buf.value + size - 16),
                                              C.byref(tc), C.byref(lost))
        assert st == pic.PIC_ERR_INVALID_ARG and "final_stock" in pic.pic_last_error()
    finally:
        rt.cudaFree(buf)
    with pytest.raises(ValueError):
        pic.pic_simulate_sequential_static(desc, "greedy", act[:10])
