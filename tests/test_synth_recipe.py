"""The seeded input recipe (paper_2406_01939_b300.synth) against what it states.

Both the oracle and the CUDA path consume these generators, so a wrong draw would
pass every parity test: here each workload's shapes, ranges and seeding are
checked, the Zipf(1.1) product mix and the Poisson stock (Sec. 4.1's
heavy-tailed demand, about 1.05x the expected demand in stock) against their
stated parameters, node capacity and the uniform assignment against their
totals and ranges, the BF16 rounding against torch's round-to-nearest-even
conversion, and the OWMR demand gaps against a brute-force scan."""
import numpy as np
import pytest
import torch

from paper_2406_01939_b300 import synth


def test_bf16_rounding_is_nearest_even():
    rng = np.random.default_rng(3)
    x = np.concatenate([
        rng.normal(0, 0.02, 20000), rng.normal(0, 1e4, 5000), rng.uniform(-3, 3, 5000),
        np.ldexp(rng.uniform(1, 2, 1000), -130),  # subnormal FP32 inputs
        [0.0, -0.0, 1.0, -1.0, 3.4e38, -3.4e38],
    ]).astype(np.float32)
    # exact ties: the low 16 bits 0x8000, both parities of the kept bit
    ties = (np.arange(2000, dtype=np.uint32) << 16 | 0x8000).astype(np.uint32) + np.uint32(0x3F800000)
    x = np.concatenate([x, ties.view(np.float32)])
    got = synth.f32_to_bf16(x)
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(got, want)
    # BF16 values survive the round trip
    np.testing.assert_array_equal(synth.f32_to_bf16(synth.bf16_to_f32(got)), got)


def test_generic_instance_shapes_ranges_and_seeding():
    a = synth.make_instance(5000, 16, 300, 40, seed=7, stock="poisson", with_lam=True)
    b = synth.make_instance(5000, 16, 300, 40, seed=7, stock="poisson", with_lam=True)
    c = synth.make_instance(5000, 16, 300, 40, seed=8, stock="poisson", with_lam=True)
    for k in ("prod", "reg", "x0", "cost", "lam"):
        va = getattr(a, k)
        assert va.dtype == np.int32 and va.flags.c_contiguous, k
        np.testing.assert_array_equal(va, getattr(b, k))  # same seed, same draw
    assert not np.array_equal(a.prod, c.prod) and not np.array_equal(a.cost, c.cost)
    assert a.prod.shape == (5000,) and a.reg.shape == (5000,)
    assert a.x0.shape == (300, 16) and a.lam.shape == (300, 16) and a.cost.shape == (40, 16)
    assert a.prod.min() >= 0 and a.prod.max() < 300 and a.reg.min() >= 0 and a.reg.max() < 40
    assert a.cost.min() >= 1 and a.cost.max() <= 100 and a.lam.min() >= 0 and a.lam.max() <= 30
    assert a.x0.min() >= 0 and a.cap is None
    u = synth.make_instance(3000, 8, 16, 32, seed=1, stock="uniform", stock_hi=20)
    assert u.x0.min() >= 0 and u.x0.max() <= 20 and u.lam is None
    assert set(np.unique(u.x0)) == set(range(21))  # every level of U{0..20} drawn
    with pytest.raises(ValueError):
        synth.make_instance(10, 2, 2, 2, stock="gamma")


def test_zipf_product_mix():
    K, T = 10_000, 1 << 18
    p = synth.zipf_probs(K, 1.1)
    assert p.sum() == pytest.approx(1.0, abs=1e-12)
    np.testing.assert_allclose(p[1:] / p[:-1], (np.arange(1, K) / np.arange(2, K + 1)) ** 1.1, rtol=1e-12)
    inst = synth.make_instance(T, 4, K, 10, seed=2, stock="uniform")
    cnt = np.bincount(inst.prod, minlength=K)
    # the 50 most popular products: each count within 5 binomial sigmas of T p_k
    mu = T * p[:50]
    assert np.all(np.abs(cnt[:50] - mu) <= 5 * np.sqrt(mu * (1 - p[:50])))
    # and the tail as a whole
    tail = cnt[1000:].sum()
    mt = T * p[1000:].sum()
    assert abs(tail - mt) <= 5 * np.sqrt(mt)
    # regions uniform
    rc = np.bincount(inst.reg, minlength=10)
    assert np.all(np.abs(rc - T / 10) <= 5 * np.sqrt(T / 10))


def test_poisson_stock_is_fill_times_expected_demand():
    T, N, K = 1 << 16, 32, 500
    inst = synth.make_instance(T, N, K, 8, seed=4, stock="poisson", fill=1.05)
    p = synth.zipf_probs(K)
    # x0[k, :] sums to Poisson(1.05 T p_k): the network stock of product k
    tot = inst.x0.sum(axis=1).astype(np.float64)
    mean = 1.05 * T * p
    z = (tot - mean) / np.sqrt(mean)
    assert np.abs(z).max() < 6 and abs(z.mean()) < 0.2 and 0.8 < z.std() < 1.2
    # spread evenly over warehouses: per-warehouse means of the top product
    assert inst.x0[0].mean() == pytest.approx(1.05 * T * p[0] / N, rel=0.05)


def test_named_workloads():
    d = synth.dual_large(0, T=1 << 14)
    assert (d.N, d.K, d.R) == (64, 10_000, 1_000) and d.lam is not None and d.cap is None
    inst, mlp = synth.mlp_medium(0, T=1 << 12)
    assert (inst.N, inst.K, inst.R) == (64, 2_000, 500) and inst.lam is None
    assert mlp.W1.shape == (2 * 64 + synth.EMB, synth.HIDDEN) and mlp.W2.shape == (synth.HIDDEN, 64)
    assert mlp.b1.shape == (synth.HIDDEN,) and mlp.b2.shape == (64,) and mlp.E.shape == (500, synth.EMB)
    w = synth.bf16_to_f32(mlp.W1)
    assert w.std() == pytest.approx(0.02, rel=0.05) and abs(w.mean()) < 1e-3
    g = synth.greedy_small(0)
    assert (g.T, g.N, g.K, g.R) == (4096, 8, 16, 32) and g.x0.max() <= 20
    c = synth.capacity_large(0, T=1 << 14)
    np.testing.assert_array_equal(c.prod, d.prod)  # dual_large's orders plus capacity
    assert c.cap.shape == (64,) and c.cap.dtype == np.int32


def test_batch_and_pg_workloads():
    insts, pols = synth.batch_uneven(0, B=6, Tlo=100, Thi=400, K=50, R=20)
    assert len(insts) == 6
    for b, (i, p) in enumerate(zip(insts, pols)):
        assert 100 <= i.T <= 400 and i.N == 32
        assert p.kind == ("greedy" if b % 2 == 0 else "mlp")
        np.testing.assert_array_equal(i.cost, insts[0].cost)  # one shared cost table
        assert i.lam is None
    assert len({i.T for i in insts}) > 1  # uneven horizons
    assert not np.array_equal(insts[0].prod[:100], insts[1].prod[:100])  # own orders
    assert pols[1].mlp is pols[3].mlp
    pinsts, mlp = synth.pg_large(0, B=3, T=256, K=40, R=10)
    assert [i.T for i in pinsts] == [256] * 3 and mlp.W2.shape == (synth.HIDDEN, 64)
    np.testing.assert_array_equal(pinsts[1].cost, pinsts[2].cost)


def test_capacity_and_assignment():
    T, N = 1 << 16, 64
    cap = synth.node_capacity(T, N, seed=1, frac=0.8)
    assert cap.dtype == np.int32 and cap.min() >= 0
    assert 0.8 * T - N <= cap.sum() <= 0.8 * T  # floors of the pro-rata shares
    assert cap.max() > cap.min()  # log-normal weights, not uniform
    P = 4096
    proc = synth.uniform_assignment(T, P, seed=2)
    assert proc.dtype == np.int32 and proc.min() >= 0 and proc.max() < P
    cnt = np.bincount(proc, minlength=P)
    chi2 = ((cnt - T / P) ** 2 / (T / P)).sum()
    assert abs(chi2 - (P - 1)) < 6 * np.sqrt(2 * (P - 1))
    np.testing.assert_array_equal(proc, synth.uniform_assignment(T, P, seed=2))


def test_owmr_recipe():
    w = synth.owmr_store_weights(50, 0.01)
    assert w.sum() == pytest.approx(1.0) and np.allclose(w[1:] / w[:-1], 0.99)
    assert np.allclose(synth.owmr_store_weights(7), 1 / 7)
    inst = synth.make_owmr(5200, 30, seed=3)
    assert inst.s == 1_000 and inst.S == 1_000 + 5200 // 52 and inst.X0 == inst.S
    assert np.all(inst.dem == 1) and np.all(inst.x0r == inst.Sl)
    assert np.all(inst.Sl <= inst.cap) and np.all(inst.sl < inst.Sl)
    small = synth.make_owmr(4000, 10, seed=4, demand="small")
    assert set(np.unique(small.dem)) == {0, 1, 2, 3}
    base, net = synth.owmr_base(0, T=20_000, N=400)
    assert (base.s, base.S) == (1_000, 71_000) and net.W2.shape == (512, 512) and net.W1.shape == (3, 512)
    with pytest.raises(ValueError):
        synth.make_owmr(10, 2, demand="poisson")


def test_demand_gaps_brute_force():
    rng = np.random.default_rng(9)
    ret = rng.integers(0, 7, size=3000).astype(np.int32)
    got = synth.demand_gaps(ret)
    last = {}
    for t, r in enumerate(ret.tolist()):
        want = t - last[r] if r in last else t + 1
        assert got[t] == min(want, 32_767), t
        last[r] = t
    # the cap: a store seen at step 0 and again 40,000 steps later
    ret = np.zeros(40_001, np.int32)
    ret[1:40_000] = 1
    g = synth.demand_gaps(ret)
    assert g[0] == 1 and g[40_000] == 32_767 and g[2] == 1
