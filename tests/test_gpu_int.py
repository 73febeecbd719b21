"""GPU parity of the integer-policy path (greedy, bid-price) against the CPU
oracle, through the C ABI.  Integer outputs are compared bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import paper_2406_01939_b300 as pic
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.session import DeviceInstance
from paper_2406_01939_b300.synth import Instance, Policy

pytestmark = pytest.mark.gpu


def rand_inst(rng, T, N, K, R, xmax=6, cmax=9, lam=True):
    return Instance(T, N, K, R,
                    rng.integers(0, K, T).astype(np.int32), rng.integers(0, R, T).astype(np.int32),
                    rng.integers(0, xmax + 1, (K, N)).astype(np.int32),
                    rng.integers(1, cmax + 1, (R, N)).astype(np.int32),
                    rng.integers(0, 4, (K, N)).astype(np.int32) if lam else None)


def check_against_oracle(inst, kind, M, dev=None, **kw):
    pol = Policy(kind)
    want = oracle.picard_chunked(inst, pol, M)
    seq = oracle.seq_sim(inst, pol)
    d = dev or DeviceInstance(inst)
    got = d.simulate(pol, "picard", num_chunks=M, **kw)
    a = got["actions"].cpu().numpy()
    np.testing.assert_array_equal(a, seq["actions"])
    np.testing.assert_array_equal(a, want["actions"])
    assert got["iters"] == want["iters"], (got["iters"], want["iters"])
    assert got["total_cost"] == seq["total_cost"]
    assert got["lost"] == seq["lost"]
    np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])
    return got, want


def test_greedy_small_workload_bit_exact():
    """T=4,096, N=8, K=16, R=32, 64 chunks: actions, cost, lost sales, final
    stock and the pass count of Algorithm 1 equal the oracle's."""
    inst = synth.greedy_small(0)
    got, want = check_against_oracle(inst, "greedy", 64)
    assert got["num_chunks"] == 64


def test_every_iterate_matches_algorithm_1():
    """Capping the passes at k returns alpha^k (status NOT_CONVERGED before the
    fixed point); every iterate equals the oracle's alpha^k."""
    inst = synth.greedy_small(1)
    pol = Policy("greedy")
    want = oracle.picard_literal(inst, pol, 64, record=True)
    d = DeviceInstance(inst)
    for k in range(1, want["iters"] + 1):
        got = d.simulate(pol, "picard", num_chunks=64, max_iters=k, raise_on_error=False)
        expect_status = pic.PIC_OK if k == want["iters"] else pic.PIC_ERR_NOT_CONVERGED
        assert got["status"] == expect_status
        np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["iterates"][k - 1])


def test_no_reset_flag_same_result_more_work():
    inst = synth.greedy_small(2)
    d = DeviceInstance(inst)
    a = d.simulate(Policy("greedy"), num_chunks=64)
    b = d.simulate(Policy("greedy"), num_chunks=64, flags=pic.PIC_FLAG_NO_RESET)
    assert torch.equal(a["actions"], b["actions"]) and a["iters"] == b["iters"]
    assert b["policy_calls"] == inst.T * b["iters"]
    assert a["policy_calls"] <= b["policy_calls"]


@pytest.mark.parametrize("N", [1, 5, 32, 33, 64, 100, 127])
def test_random_shapes_and_ragged_lanes(N):
    rng = np.random.default_rng(N)
    for T, K, R in ((0, 3, 2), (1, 1, 1), (2, 2, 3), (37, 4, 5), (1000, 300, 7), (5000, 17, 40)):
        inst = rand_inst(rng, T, N, K, R)
        dev = DeviceInstance(inst)
        for kind in ("greedy", "dual"):
            for M in sorted({1, 7, max(1, T)}):
                for W in (1, 3, 64):
                    for flags in (0, pic.PIC_FLAG_GROUP_KERNEL):
                        check_against_oracle(inst, kind, M, dev=dev, seg_window=W, flags=flags)


def test_wide_costs_use_global_table():
    """Costs beyond int16 (no shared-memory table): same bit-exact results."""
    rng = np.random.default_rng(11)
    for N in (8, 40, 64):
        inst = rand_inst(rng, 3000, N, 20, 9, xmax=8, cmax=9)
        inst.cost = (inst.cost.astype(np.int64) * 100_003 - 300_000).astype(np.int32)
        inst.lam = (inst.lam.astype(np.int64) * 99_991).astype(np.int32)
        dev = DeviceInstance(inst)
        for kind in ("greedy", "dual"):
            for M in (1, 30, 3000):
                check_against_oracle(inst, kind, M, dev=dev)


def test_sequential_mode_bit_exact():
    rng = np.random.default_rng(5)
    for inst in (synth.greedy_small(3), rand_inst(rng, 3000, 64, 50, 20), rand_inst(rng, 777, 100, 9, 3),
                 rand_inst(rng, 1, 1, 1, 1)):
        d = DeviceInstance(inst)
        for kind in ("greedy", "dual") if inst.lam is not None else ("greedy",):
            seq = oracle.seq_sim(inst, Policy(kind))
            got = d.simulate(Policy(kind), "sequential")
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
            assert got["total_cost"] == seq["total_cost"] and got["lost"] == seq["lost"]
            assert got["iters"] == 1
            np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), seq["x_final"])


def test_warm_start_cache():
    """Any initial cache converges to the sequential path (proof of Prop. 1 does
    not use alpha^0); pass count equals the oracle's from the same cache."""
    rng = np.random.default_rng(6)
    inst = rand_inst(rng, 4000, 16, 30, 12)
    d = DeviceInstance(inst)
    for kind in ("greedy", "dual"):
        pol = Policy(kind)
        seq = oracle.seq_sim(inst, pol)
        for init in (rng.integers(-1, 16, inst.T).astype(np.int8), seq["actions"]):
            want = oracle.picard_chunked(inst, pol, 40, alpha_init=init)
            got = d.simulate(pol, num_chunks=40, alpha_init=init)
            np.testing.assert_array_equal(got["actions"].cpu().numpy(), seq["actions"])
            assert got["iters"] == want["iters"]
        # the sequential path itself is a fixed point: one confirming pass
        assert d.simulate(pol, num_chunks=40, alpha_init=seq["actions"])["iters"] == 1


def test_invalid_inputs_rejected():
    rng = np.random.default_rng(7)
    inst = rand_inst(rng, 100, 4, 3, 2)
    bad = Instance(inst.T, inst.N, inst.K, inst.R, inst.prod.copy(), inst.reg, inst.x0, inst.cost, inst.lam)
    bad.prod[5] = 3  # == K
    with pytest.raises(pic.PicError) as e:
        DeviceInstance(bad)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG
    neg = Instance(inst.T, inst.N, inst.K, inst.R, inst.prod, inst.reg, -inst.x0 - 1, inst.cost, inst.lam)
    with pytest.raises(pic.PicError):
        DeviceInstance(neg)
    nolam = Instance(inst.T, inst.N, inst.K, inst.R, inst.prod, inst.reg, inst.x0, inst.cost, None)
    d = DeviceInstance(nolam)
    with pytest.raises(pic.PicError) as e:
        d.simulate(Policy("dual"))
    assert e.value.status == pic.PIC_ERR_INVALID_ARG
    d2 = DeviceInstance(inst)
    with pytest.raises(pic.PicError) as e:
        d2.simulate(Policy("greedy"), alpha_init=np.full(inst.T, 9, np.int8))
    assert e.value.status == pic.PIC_ERR_INVALID_ARG
    # the instance still works after the rejected call
    check_against_oracle(inst, "greedy", 10, dev=d2)


def test_timeout_reports_error_and_context_survives():
    """A 1 ns bound on device-side waits makes the first grid barrier give up:
    the call returns PIC_ERR_TIMEOUT and the next call on the same context works."""
    inst = synth.greedy_small(4)
    d = DeviceInstance(inst)
    got = d.simulate(Policy("greedy"), num_chunks=64, timeout_ns=1, raise_on_error=False)
    assert got["status"] == pic.PIC_ERR_TIMEOUT
    check_against_oracle(inst, "greedy", 64, dev=d)


def test_host_buffers_end_to_end():
    """Host input arrays and host output buffers through the same ABI."""
    inst = synth.greedy_small(8)
    d = DeviceInstance(inst)
    inst2 = synth.greedy_small(9)
    host = {k: np.ascontiguousarray(getattr(inst2, k), np.int32) for k in ("prod", "reg", "x0", "cost")}
    host["lam"] = None
    d.inst = inst2
    d.load_host(host)
    act = np.empty(inst2.T, np.int8)
    stock = np.empty((inst2.K, inst2.N), np.int32)
    opts = pic.make_opts("picard", 64, out_mem=pic.PIC_MEM_HOST)
    st, res = pic.pic_simulate(d.handle, pic.make_policy("greedy"), opts, act, stock)
    seq = oracle.seq_sim(inst2, Policy("greedy"))
    np.testing.assert_array_equal(act, seq["actions"])
    np.testing.assert_array_equal(stock, seq["x_final"])
    assert res.total_cost == seq["total_cost"]


@pytest.mark.parametrize("M", [256, 4096, 65536])
def test_dual_large_full_size(M):
    """T=2^20, N=64, K=10,000, R=1,000 bid-price workload (the benchmark's
    shape): bit-exact fixed point and the oracle's pass count, both layouts."""
    inst = synth.dual_large(0)
    dev = DeviceInstance(inst)
    check_against_oracle(inst, "dual", M, dev=dev)
    check_against_oracle(inst, "dual", M, dev=dev, flags=pic.PIC_FLAG_GROUP_KERNEL)


def test_pass_trace_records_every_pass():
    """The per-pass trace has one row per pass: increasing timestamps, and its
    policy-call column sums to the call's total; the largest unit of a pass made
    at most the pass's calls and walked at least its own calls' orders."""
    inst = synth.greedy_small(5)
    d = DeviceInstance(inst)
    tr = np.zeros((100, 6), np.int64)
    got = d.simulate(Policy("greedy"), num_chunks=64, trace=tr)
    n = got["iters"]
    assert (tr[n:] == 0).all()
    stamps = tr[:n, :2].reshape(-1)
    assert (np.diff(stamps) >= 0).all() and stamps[0] > 0
    assert tr[:n, 2].sum() == got["policy_calls"]
    assert tr[:n, 3].sum() == got["seg_replays"]
    assert tr[0, 2] == inst.T  # every order is evaluated in the first pass
    assert (tr[:n, 4] <= tr[:n, 2]).all() and (tr[:n, 4] <= tr[:n, 5]).all()
    assert ((tr[:n, 4] > 0) == (tr[:n, 2] > 0)).all()


def test_reused_order_tables_equal_rebuilt_ones():
    """PIC_FLAG_REUSE_TABLES keeps the order tables of an earlier call with the
    same chunk count and segment window: the result equals the oracle's after
    calls in other modes, other chunkings, other policies and a reload of the
    inputs (which invalidates the tables)."""
    R = pic.PIC_FLAG_REUSE_TABLES
    inst = synth.dual_large(2, T=1 << 15, K=900, R=80)
    d = DeviceInstance(inst)
    check_against_oracle(inst, "dual", 256, dev=d)
    for kind in ("dual", "greedy"):
        check_against_oracle(inst, kind, 256, dev=d, flags=R)
    check_against_oracle(inst, "dual", 512, dev=d, flags=R)  # other chunking: rebuilt
    check_against_oracle(inst, "dual", 512, dev=d, flags=R, seg_window=8)
    d.simulate(Policy("dual"), "sequential")
    d.simulate(Policy("dual"), "products", num_chunks=300)
    d.simulate(Policy("dual"), "assigned", num_chunks=64,
               proc=torch.as_tensor(synth.uniform_assignment(inst.T, 64, seed=1)).cuda())
    check_against_oracle(inst, "dual", 512, dev=d, flags=R, seg_window=8)
    # max_steps window with kept tables
    want = oracle.picard_windowed(inst, Policy("dual"), 512, 4096)
    got = d.simulate(Policy("dual"), "picard", num_chunks=512, seg_window=8, max_steps=4096, flags=R)
    np.testing.assert_array_equal(got["actions"].cpu().numpy(), want["actions"])
    assert got["iters"] == want["iters"]
    # new inputs of the same shape: the tables are rebuilt
    inst2 = synth.dual_large(3, T=1 << 15, K=900, R=80)
    d.inst = inst2
    d.load_host({k: np.ascontiguousarray(getattr(inst2, k), np.int32)
                 for k in ("prod", "reg", "x0", "cost", "lam")})
    check_against_oracle(inst2, "dual", 512, dev=d, flags=R, seg_window=8)
