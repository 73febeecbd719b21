"""Batched simulation (pic_create_batch / pic_simulate_batch) on the GPU against
the CPU oracle, trajectory by trajectory: actions, final stock, cost, a^phi
count and each trajectory's own Picard pass count must be identical to what the
oracle computes for that trajectory alone with the same chunk count."""
import numpy as np
import pytest
import torch

import oracle
import paper_2406_01939_b300 as pic
from paper_2406_01939_b300 import synth
from paper_2406_01939_b300.session import DeviceBatch
from paper_2406_01939_b300.synth import Policy

pytestmark = pytest.mark.gpu

KINDS = ("greedy", "dual", "mlp", "gumbel")


def mixed_batch(seed, Ts, N, K=12, R=9, kinds=KINDS):
    """Trajectories with their own sizes, stock and tables; policies cycle
    through `kinds`; one MLP parameter set (E has R rows: every trajectory uses
    the same R)."""
    rng = np.random.default_rng(seed)
    mlp = synth.make_mlp(N, R, seed=seed)
    insts, pols = [], []
    for b, T in enumerate(Ts):
        Kb = int(rng.integers(1, K + 1))
        inst = synth.make_instance(int(T), N, Kb, R, seed=1000 * seed + b, stock="poisson",
                                   fill=0.9, with_lam=True)
        kind = kinds[b % len(kinds)]
        insts.append(inst)
        pols.append(Policy(kind, mlp=mlp if kind in ("mlp", "gumbel") else None,
                           seed=77 + b, traj=b))
    return insts, pols


def check_against_oracle(db, insts, pols, got, M=None, cache=None):
    """cache: a dict kept across calls on the same trajectories and policies,
    holding the oracle's results (its sequential path; its pass count per M)."""
    cache = {} if cache is None else cache
    acts = got["actions"]
    acts = acts.cpu().numpy() if torch.is_tensor(acts) else acts
    stock = got["final_stock"]
    stock = stock.cpu().numpy() if torch.is_tensor(stock) else stock
    tot_c = tot_l = 0
    for b, (inst, pol) in enumerate(zip(insts, pols)):
        key = (b, id(inst), id(pol))
        if key not in cache:
            cache[key] = oracle.seq_sim(inst, pol)
        want = cache[key]
        np.testing.assert_array_equal(db.split(acts)[b], want["actions"], err_msg=f"traj {b}")
        np.testing.assert_array_equal(db.split_stock(stock)[b], want["x_final"], err_msg=f"traj {b}")
        tr = got["traj"][b]
        assert tr["total_cost"] == want["total_cost"] and tr["lost"] == want["lost"], b
        assert tr["converged"] == 1
        if M is not None and inst.T > 0:
            if key + (M,) not in cache:
                cache[key + (M,)] = oracle.picard_chunked(inst, pol, M)["iters"]
            assert tr["iters"] == cache[key + (M,)], b
        tot_c += want["total_cost"]
        tot_l += want["lost"]
    assert got["total_cost"] == tot_c and got["lost"] == tot_l


@pytest.mark.parametrize("N", [8, 32, 33])
def test_batch_mixed_policies_match_oracle(N):
    Ts = [0, 1, 37, 300, 1000, 1500, 64, 777, 2000]
    insts, pols = mixed_batch(N, Ts, N)
    db = DeviceBatch(insts)
    cache = {}
    for M in (1, 7, 40):
        got = db.simulate(pols, "picard", num_chunks=M)
        check_against_oracle(db, insts, pols, got, M, cache)
        assert got["iters"] == max(t["iters"] for t in got["traj"])


def test_batch_sequential_mode_matches_oracle():
    insts, pols = mixed_batch(5, [500, 3, 1200, 0, 900, 250, 1800], 16)
    db = DeviceBatch(insts)
    got = db.simulate(pols, "sequential")
    check_against_oracle(db, insts, pols, got)
    assert all(t["iters"] == 1 for t in got["traj"])


def test_batch_iterates_equal_oracle_iterates():
    """With max_iters = k every trajectory's cache equals the oracle's alpha^k."""
    insts, pols = mixed_batch(11, [400, 900, 650, 1200], 8)
    db = DeviceBatch(insts)
    M = 12
    want = [oracle.picard_chunked(i, p, M, record=True) for i, p in zip(insts, pols)]
    for k in (1, 2, 3, 5):
        got = db.simulate(pols, "picard", num_chunks=M, max_iters=k, raise_on_error=False)
        a = got["actions"].cpu().numpy()
        for b in range(len(insts)):
            kk = min(k, want[b]["iters"])
            np.testing.assert_array_equal(db.split(a)[b], want[b]["iterates"][kk - 1],
                                          err_msg=f"traj {b} pass {k}")


def test_batch_graph_relaunch_and_policy_change():
    """PIC_FLAG_GRAPH: the captured graph is relaunched with new per-trajectory
    policies (kinds, seeds) and still gives the oracle's paths."""
    insts, pols = mixed_batch(3, [800, 1300, 500, 950, 1100, 60], 24)
    db = DeviceBatch(insts)
    M = 16
    flags = pic.PIC_FLAG_GRAPH | pic.PIC_FLAG_TIMING
    g1 = db.simulate(pols, "picard", num_chunks=M, flags=flags)
    check_against_oracle(db, insts, pols, g1, M)
    g2 = db.simulate(pols, "picard", num_chunks=M, flags=flags)  # relaunch, tables kept
    g2b = db.simulate(pols, "picard", num_chunks=M, flags=flags)
    assert torch.equal(g1["actions"], g2["actions"]) and torch.equal(g1["actions"], g2b["actions"])
    assert g2["launches"] == g2b["launches"] < g1["launches"]  # g1 also built the tables
    assert g1["iters"] == g2["iters"] == g2b["iters"]
    mlp = next(p.mlp for p in pols if p.mlp is not None)
    swapped = [Policy("mlp", mlp=mlp, seed=p.seed, traj=p.traj) if p.kind == "greedy" else
               (Policy("gumbel", mlp=mlp, seed=p.seed + 5, traj=p.traj) if p.kind == "gumbel" else p)
               for p in pols]
    g3 = db.simulate(swapped, "picard", num_chunks=M, flags=flags)
    check_against_oracle(db, insts, swapped, g3, M)
    # a different chunk count is a different graph
    g4 = db.simulate(swapped, "picard", num_chunks=M + 3, flags=flags)
    check_against_oracle(db, insts, swapped, g4, M + 3)


def test_batch_tensor_core_tiles_exact():
    """PIC_FLAG_TC in a batch: MLP and Gumbel trajectories with long runs and
    ample stock use the tensor-core tiles; results are the oracle's."""
    Ts = [6000, 9000, 4000, 7000, 5000, 8000]
    insts, pols = mixed_batch(31, Ts, 32, K=5, R=9)
    for i in insts:
        i.x0 = (i.x0 * 40 + 50).astype(np.int32)  # ample stock: features saturate
    db = DeviceBatch(insts)
    got = db.simulate(pols, "picard", num_chunks=3, flags=pic.PIC_FLAG_TC | pic.PIC_FLAG_NO_SAT)
    check_against_oracle(db, insts, pols, got, 3)
    assert got["tc_decisions"] > 0


def test_batch_autotuner_choice_is_exact():
    insts, pols = mixed_batch(8, [3000, 2500, 4000, 1000, 3500, 2000, 1800, 2600], 32)
    db = DeviceBatch(insts)
    got = db.simulate(pols, "picard", num_chunks=0)
    M = got["num_chunks"]
    assert M >= 1 and got["seg_window"] >= 1 and got["cta_threads"] in (256, 512)
    check_against_oracle(db, insts, pols, got, M)
    again = db.simulate(pols, "picard", num_chunks=0)  # cached choice
    assert again["num_chunks"] == M and again["seg_window"] == got["seg_window"]
    assert torch.equal(again["actions"], got["actions"])


def test_batch_host_outputs_and_integer_only():
    insts, pols = mixed_batch(21, [700, 1400, 900], 40, kinds=("greedy", "dual"))
    db = DeviceBatch(insts, mem=pic.PIC_MEM_HOST)
    got = db.simulate(pols, "picard", num_chunks=9, out_mem=pic.PIC_MEM_HOST)
    assert isinstance(got["actions"], np.ndarray)
    check_against_oracle(db, insts, pols, got, 9)


def test_batch_invalid_inputs():
    insts, pols = mixed_batch(2, [100, 200], 8)
    with pytest.raises(pic.PicError) as e:
        DeviceBatch([insts[0], synth.make_instance(50, 9, 4, 9, seed=1)])
    assert e.value.status == pic.PIC_ERR_INVALID_ARG and "N" in str(e.value)
    bad = synth.make_instance(50, 8, 4, 9, seed=1)
    bad.prod = bad.prod.copy()
    bad.prod[7] = 4  # K = 4
    with pytest.raises(pic.PicError) as e:
        DeviceBatch([insts[0], bad])
    assert e.value.status == pic.PIC_ERR_INVALID_ARG and "prod" in str(e.value)
    db = DeviceBatch(insts)
    two = [Policy("mlp", mlp=synth.make_mlp(8, 9, seed=98)),
           Policy("mlp", mlp=synth.make_mlp(8, 9, seed=99))]  # two weight sets
    with pytest.raises(pic.PicError) as e:
        db.simulate(two, "picard", num_chunks=4)
    assert e.value.status == pic.PIC_ERR_UNSUPPORTED
    nolam = [synth.make_instance(80, 8, 3, 9, seed=4), synth.make_instance(90, 8, 3, 9, seed=5)]
    db2 = DeviceBatch(nolam)
    with pytest.raises(pic.PicError) as e:
        db2.simulate([Policy("greedy"), Policy("dual")], "picard", num_chunks=4)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG and "lam" in str(e.value)


def test_batch_uneven_full_size():
    """512 trajectories, T_b ~ U{16,384..262,144}, N=32, K=2,000, R=200, even
    index greedy, odd index MLP: one persistent launch (autotuned, run as a CUDA
    graph) equals the batched sequential simulation trajectory by trajectory, and
    the first greedy and the first MLP trajectory, whole, equal the oracle's
    sequential simulation (every action, final stock, cost, lost count)."""
    insts, pols = synth.batch_uneven(0)
    db = DeviceBatch(insts)
    flags = pic.PIC_FLAG_GRAPH
    got = db.simulate(pols, "picard", num_chunks=0, flags=flags)
    seq = db.simulate(pols, "sequential")
    assert torch.equal(got["actions"], seq["actions"])
    assert torch.equal(got["final_stock"], seq["final_stock"])
    for b in range(len(insts)):
        assert got["traj"][b]["total_cost"] == seq["traj"][b]["total_cost"], b
        assert got["traj"][b]["lost"] == seq["traj"][b]["lost"], b
        assert got["traj"][b]["converged"] == 1
    a = db.split(got["actions"].cpu().numpy())
    xf = db.split_stock(got["final_stock"].cpu().numpy())
    for b in (0, 1):  # greedy, MLP
        want = oracle.seq_sim(insts[b], pols[b])
        np.testing.assert_array_equal(a[b], want["actions"], err_msg=f"trajectory {b}")
        np.testing.assert_array_equal(xf[b], want["x_final"])
        assert got["traj"][b]["total_cost"] == want["total_cost"], b
        assert got["traj"][b]["lost"] == want["lost"], b


def test_batch_saturated_table_exact():
    """The saturated-state score table in a batch (one table over the combined
    regions): Picard and batched sequential runs equal the oracle with and
    without it."""
    insts, pols = mixed_batch(41, [3000, 2500, 4000, 1500], 32, K=6, R=9)
    for i in insts:
        i.x0 = (i.x0 + 40).astype(np.int32)  # saturated for a while
    db = DeviceBatch(insts)
    cache = {}
    for flags in (0, pic.PIC_FLAG_NO_SAT):
        for mode in ("picard", "sequential"):
            got = db.simulate(pols, mode, num_chunks=9, flags=flags)
            check_against_oracle(db, insts, pols, got, 9 if mode == "picard" else None, cache)
            assert (got["sat_decisions"] > 0) == (flags == 0)


def test_batch_load_replaces_the_inputs():
    """pic_batch_load: a batch created from one set of trajectories and then
    loaded with a second set of the same shapes simulates the second set as the
    oracle does, through rebuilt order tables and a recaptured graph; a load
    that fails a range check leaves the batch refusing calls until a valid one."""
    N = 32
    insts, pols = mixed_batch(5, [300, 1200, 50, 900, 700], N)
    fresh = [synth.make_instance(i.T, N, i.K, i.R, seed=4242 + b, stock="poisson", fill=0.9,
                                 with_lam=True) for b, i in enumerate(insts)]
    db = DeviceBatch(insts)
    for flags in (0, pic.PIC_FLAG_GRAPH):  # tables (and a graph) of the first set
        check_against_oracle(db, insts, pols, db.simulate(pols, "picard", num_chunks=16, flags=flags))
    db.load(fresh, mem=pic.PIC_MEM_HOST)
    for flags in (pic.PIC_FLAG_GRAPH, 0):
        check_against_oracle(db, fresh, pols, db.simulate(pols, "picard", num_chunks=16, flags=flags), M=16)
    bad = [synth.make_instance(i.T, N, i.K, i.R, seed=77 + b, with_lam=True) for b, i in enumerate(insts)]
    bad[3].prod = bad[3].prod.copy()
    bad[3].prod[5] = bad[3].K  # out of range
    with pytest.raises(pic.PicError) as e:
        db.load(bad)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG and "prod" in str(e.value)
    with pytest.raises(pic.PicError) as e:
        db.simulate(pols, "picard", num_chunks=16)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG and "pic_batch_load" in str(e.value)
    with pytest.raises(pic.PicError) as e:
        db.load(fresh[:-1])  # one trajectory short
    assert e.value.status == pic.PIC_ERR_INVALID_ARG
    other = list(fresh)
    other[1] = synth.make_instance(fresh[1].T + 1, N, fresh[1].K, fresh[1].R, seed=3, with_lam=True)
    with pytest.raises(pic.PicError) as e:
        db.load(other)
    assert e.value.status == pic.PIC_ERR_INVALID_ARG and "trajectory 1" in str(e.value)
    db.load(insts)  # device arrays; back to the first set
    check_against_oracle(db, insts, pols, db.simulate(pols, "picard", num_chunks=16), M=16)
