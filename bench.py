#!/usr/bin/env python
"""Benchmark: orders simulated per second by Picard iteration (Algorithm 1) on
one B300, against the sequential GPU simulator, bit-exact.

A step is one whole simulation of one synthetic trajectory from its order
stream resident in HBM: the product-major order tables (sort, runs, segments),
every Picard pass to the fixed point, and the outputs (actions in time order,
total cost).  Default workload (bid-price FO, the large single-trajectory
shape): T = 2^20 orders, N = 64 warehouses, K = 10,000 products (Zipf 1.1
demand), R = 1,000 regions, stock ~ Poisson(1.05 T p_k / N), M = 4,096 time
chunks.  --workload mlp_medium: T = 2^18, N = 64, K = 2,000, R = 500, MLP
policy.  --workload batch_uneven: 512 trajectories of T_b ~ U{16,384..262,144}
orders, N = 32, K = 2,000, R = 200, even index greedy, odd index MLP, one
persistent launch per step (autotuned chunking, CUDA graph).  --workload
pg_large: a policy-gradient step over 64 trajectories of T = 2^20 orders (N = 64,
K = 10,000, R = 1,000, Gumbel-max MLP): the batch simulated by Picard, then the
REINFORCE gradient (hand-written backward kernel).  --workload owmr_base: the
OWMR inventory-control base case of Appendix B.3 (T = 3,650,000 unit demands
over 4,000 stores, central (s, S) = (1,000, 71,000), width-512 retailer
network), one processor per store, max_steps window of 80,000 steps.

Prints one JSON line (rank 0).  Under torchrun every rank simulates its own
trajectory (weak scaling, no collective on the data path).  --impl reference
times the CPU oracle (plain C sequential simulator) on the host instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "orders simulated/sec on 1 B300, Picard vs sequential GPU sim, bit-exact; iters"
UNIT = "orders/s"


def over_ranks(x, world, op="max", device=None):
    """Reduce one float over the ranks of the job (identity at world size 1).
    "max" gives the job's time from each rank's timed total (every rank starts
    after the same barrier); "sum" gives the job's units."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_this_rank, steps, t_ms_this_rank, world, device=None):
    """Whole-job throughput: the units all ranks processed in the timed steps
    over the slowest rank's time.  Returns (rate, job time in ms)."""
    t_ms = over_ranks(t_ms_this_rank, world, "max", device)
    units = over_ranks(units_this_rank * steps, world, "sum", device)
    return units / (t_ms / 1000.0), t_ms


def rank_seed(base, rank):
    """Each rank simulates its own synthetic workload (weak scaling)."""
    return base + rank


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--chunks", type=int, default=-1,
                   help="time chunks M (-1: the workload's default; 0: autotune, batch only)")
    p.add_argument("--seg-window", type=int, default=0)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--seq-steps", type=int, default=3)
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--T", type=int, default=0, help="orders (0 = the workload's own size)")
    p.add_argument("--workload", default="dual_large",
                   choices=["dual_large", "greedy_small", "mlp_medium", "batch_uneven",
                            "pg_large", "capacity_large", "owmr_base"])
    p.add_argument("--shard", default="none", choices=["none", "products"],
                   help="single-trajectory workloads under torchrun: products (one trajectory's "
                        "products over the ranks, balanced by demand; strong scaling) or none "
                        "(every rank its own trajectory; weak scaling)")
    p.add_argument("--chunk-sweep", default="",
                   help="comma-separated chunk counts: one JSON line per count (single-trajectory "
                        "workloads), e.g. 256,1024,4096,16384,65536")
    p.add_argument("--flags", type=int, default=0, help="extra pic_sim_opts flags (tuning)")
    p.add_argument("--max-steps", type=int, default=-1,
                   help="Picard window of App. A.3 in orders (-1: the workload's default, 0: none)")
    p.add_argument("--fresh-tables", action="store_true",
                   help="rebuild the order tables on every timed call (single trajectories)")
    p.add_argument("--partition", default="chunks", choices=["chunks", "products", "random"],
                   help="FO workloads: Algorithm 1 on contiguous time chunks (default), the "
                        "product partition of Sec. 3 (one processor per product), or the uniform "
                        "random assignment of Sec. 4.1 over --chunks processes (with node capacity every "
                        "process replays the horizon in its own state: give few processes)")
    p.add_argument("--skew", type=float, default=0.0,
                   help="owmr_base: store weights (1 - skew)^n (App. B.3 ablation; 0 = uniform)")
    p.add_argument("--B", type=int, default=0,
                   help="trajectories of batch_uneven / pg_large (0 = the workload's 512 / 64)")
    return p.parse_args()


# mlp_medium: the window of App. A.3 (16,384 orders = 4 chunks), short segments
DEFAULT_MAX_STEPS = {"mlp_medium": 16384, "owmr_base": 80_000}
DEFAULT_SEG_WINDOW = {"mlp_medium": 4, "greedy_small": 16}

DEFAULT_CHUNKS = {"dual_large": 4096, "greedy_small": 64, "mlp_medium": 4096, "batch_uneven": 0,
                  "pg_large": 0, "capacity_large": 16384}

# FP32 CUDA-core peak of the MLP scorer's arithmetic: 148 SMs x 128 FP32 lanes x
# 2 FLOP per FMA x 2.032 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12


def mlp_flops_per_call(N):
    """FLOPs of one MLP decision after the per-region prefix: the stock rows of
    layer 1 (N x 256 FMA) and layer 2 (256 x N FMA), 2 FLOP per FMA."""
    return 2 * (N * 256 + 256 * N)


def make_workload(args, seed):
    """(instance, policy, policy-kind name) of the named synthetic workload."""
    from paper_2406_01939_b300 import synth
    from paper_2406_01939_b300.synth import Policy
    if args.workload == "mlp_medium":
        inst, mlp = synth.mlp_medium(seed, **({"T": args.T} if args.T else {}))
        return inst, Policy("mlp", mlp=mlp), "mlp"
    if args.workload == "capacity_large":
        inst = synth.capacity_large(seed, **({"T": args.T} if args.T else {}))
        return inst, Policy("dual"), "dual"
    if args.workload == "greedy_small":
        inst = synth.greedy_small(seed, **({"T": args.T} if args.T else {}))
        return inst, Policy("greedy"), "greedy"
    inst = synth.dual_large(seed, **({"T": args.T} if args.T else {}))
    return inst, Policy("dual"), "dual"


def batch_config(args, insts, res):
    Ts = [i.T for i in insts]
    cfg = {
        "workload": "batch_uneven",
        "desc": (f"FO batch, B={len(insts)} trajectories, T_b~U{{16384..262144}} "
                 f"(total {sum(Ts)} orders), N={insts[0].N}, K={insts[0].K}, R={insts[0].R} per "
                 f"trajectory, even index greedy / odd index MLP Linear(2N+16,256)-ReLU-Linear(256,N) "
                 f"BF16 N(0,0.02), x0~Poisson(1.05 T p_k/N), cost~U{{1..100}}"),
        "B": len(insts), "T_total": int(sum(Ts)), "T_min": int(min(Ts)), "T_max": int(max(Ts)),
        "N": insts[0].N, "K": insts[0].K, "R": insts[0].R,
        "l2": "inputs (about 0.6 GB of orders) exceed L2; flushed between timed steps (256 MiB write)",
    }
    if res is not None:
        cfg.update({"chunks_per_trajectory": res["num_chunks"], "seg_window": res["seg_window"],
                    "cta_threads": res["cta_threads"], "ctas_per_sm": res["ctas_per_sm"],
                    "tuning": "autotuned" if chunks_of(args) == 0 else "fixed", "cuda_graph": True})
    return cfg


def workload_config(args, inst):
    pol = {"mlp_medium": "MLP Linear(2N+16,256)-ReLU-Linear(256,N), BF16 N(0,0.02)",
           "greedy_small": "greedy (argmin cost over stocked warehouses)"}.get(
               args.workload, "bid-price, lambda~U{0..30}")
    stock = "x0~U{0..20}" if args.workload == "greedy_small" else "x0~Poisson(1.05 T p_k/N)"
    cap = (", node capacity for 80% of the orders (log-normal(0, 0.5) node weights), chunks "
           "of 64 orders replayed in time order" if getattr(inst, "cap", None) is not None else "")
    return {
        "workload": args.workload,
        "desc": (f"FO, T={inst.T} orders, N={inst.N} warehouses, K={inst.K} products "
                 f"(Zipf 1.1), R={inst.R} regions, {stock}, cost~U{{1..100}}, "
                 f"{pol}{cap}"),
        "T": inst.T, "N": inst.N, "K": inst.K, "R": inst.R,
        "chunks": chunks_of(args) if args.partition != "products" else None,
        "partition": {"chunks": "contiguous time chunks",
                      "products": f"products (processor of product k: k mod {inst.K})",
                      "random": f"uniform random over {chunks_of(args)} processes (seeded)"}[
                          args.partition],
        "policy": {"mlp_medium": "mlp", "greedy_small": "greedy"}.get(args.workload, "dual"),
        "max_steps": (args.max_steps if args.max_steps >= 0 else
                      DEFAULT_MAX_STEPS.get(args.workload, 0)) or None,
        "l2": "flushed between timed steps (256 MiB write)",
    }


def load_bf16_peak(sustained=False):
    """Measured dense BF16 TFLOP/s: the burst figure for a kernel timed alone,
    the sustained one for a kernel timed inside a long step."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if sustained and "bf16_tflops_sustained" in d:
            return float(d["bf16_tflops_sustained"]), "measured (sustained)"
        return float(d["bf16_tflops"]), "measured"
    return (1400.0, "fallback (sustained)") if sustained else (1800.0, "fallback")


def chunks_of(args):
    return DEFAULT_CHUNKS[args.workload] if args.chunks < 0 else args.chunks


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


_KERNEL_FILES = {
    "int": ("pic_int.cu", "pic_replay.cuh", "pic_picard.cuh", "pic_device.cuh", "pic_internal.h"),
    "capacity": ("pic_cap.cu", "pic_picard.cuh", "pic_device.cuh", "pic_internal.h"),
    "mlp": ("pic_mlp.cu", "pic_mlp.cuh", "pic_picard.cuh", "pic_device.cuh", "pic_internal.h"),
    "batch": ("pic_batch.cu", "pic_mlp.cuh", "pic_replay.cuh", "pic_picard.cuh", "pic_device.cuh",
              "pic_internal.h"),
    "wave": ("pic_wave.cu", "pic_tc.cuh", "pic_mlp.cuh", "pic_device.cuh", "pic_internal.h"),
    "pg": ("pic_pg.cu", "pic_tc.cuh", "pic_device.cuh", "pic_internal.h"),
    "owmr": ("pic_owmr.cu", "pic_device.cuh"),
}
_PROFILES = {"int": "picard_int_dual_large.md", "capacity": "picard_cap_capacity_large.md",
             "mlp": "picard_mlp_mlp_medium.md", "batch": "picard_batch_batch_uneven.md",
             "wave": "picard_wave_pg_large.md", "pg": "pg_grad_pg_large.md",
             "owmr": "owmr_picard_owmr_base.md"}


def kernel_source_hash(kind="int"):
    h = hashlib.sha256()
    for f in _KERNEL_FILES[kind]:
        h.update(open(os.path.join(ROOT, "paper_2406_01939_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kind="int"):
    """DRAM bytes per launch of the Picard kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", _PROFILES[kind])
    if not os.path.exists(p):
        return None
    src = kernel_source_hash(kind)
    hash_ok, traffic = False, None
    for line in open(p):
        if line.startswith("kernel_source_hash:") and line.split(":", 1)[1].strip() == src:
            hash_ok = True
        if line.startswith("dram_bytes_per_launch:"):
            try:
                traffic = float(line.split(":", 1)[1].strip())
            except ValueError:
                traffic = None
    return traffic if hash_ok else None


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def prefix_instance(inst, T):
    """The first T orders of a trajectory (sequential simulation is causal, so its
    actions are the first T actions of the full trajectory)."""
    from paper_2406_01939_b300.synth import Instance
    sub = Instance(T, inst.N, inst.K, inst.R, inst.prod[:T].copy(), inst.reg[:T].copy(), inst.x0,
                   inst.cost, inst.lam)
    sub.cap = getattr(inst, "cap", None)
    return sub


def cpu_oracle_rate(inst, pol, seconds):
    """The CPU oracle's sequential simulator on the host (1 thread) for about
    `seconds`: the full trajectory repeated, or, when one full run would take
    longer, a prefix of the trajectory sized to the budget.
    Returns (orders/s, sample description, oracle output, orders covered)."""
    import oracle
    probe_T = min(inst.T, 2048)
    t0 = time.perf_counter()
    oracle.seq_sim(prefix_instance(inst, probe_T), pol)
    per_order = max((time.perf_counter() - t0) / probe_T, 1e-9)
    if per_order * inst.T > seconds:
        Ts = max(probe_T, min(inst.T, int(seconds / per_order)))
        sub = prefix_instance(inst, Ts)
        t0 = time.perf_counter()
        out = oracle.seq_sim(sub, pol)
        el = time.perf_counter() - t0
        return Ts / el, f"first {Ts} of {inst.T} orders, sequential C oracle, 1 thread ({el:.1f} s)", out, Ts
    n, t0 = 0, time.perf_counter()
    while True:
        out = oracle.seq_sim(inst, pol)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return (n * inst.T / el, f"full {inst.T}-order trajectory x{n} ({el:.1f} s), sequential C oracle, "
            f"1 thread", out, inst.T)


def batch_oracle_sample(insts, pols, seconds):
    """The CPU oracle on whole trajectories of a batch, in order, for about
    `seconds` (1 thread).  Returns (orders/s, sample, [(b, oracle output)])."""
    import oracle
    done, orders, t0 = [], 0, time.perf_counter()
    for b, (inst, pol) in enumerate(zip(insts, pols)):
        out = oracle.seq_sim(inst, pol)
        done.append((b, out))
        orders += inst.T
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    kinds = sorted({pols[b].kind for b, _ in done})
    return (orders / el, f"trajectories 0..{len(done) - 1} of {len(insts)} ({orders} orders, "
            f"{'/'.join(kinds)}), sequential C oracle, 1 thread ({el:.1f} s)", done)


def run_reference(args):
    import oracle
    per = max(1, int(args.steps))
    # each step a bounded sample, so that warm-up + timed steps take about a minute
    budget = max(0.05, min(10.0, 60.0 / (per + max(0, args.warmup))))
    if args.workload == "owmr_base":
        from oracle import owmr as ow
        from paper_2406_01939_b300 import synth
        inst, net = synth.owmr_base(args.seed, a=args.skew, **({"T": args.T} if args.T else {}))
        cut = lambda n: synth.OwmrInstance(n, inst.N, inst.ret[:n], inst.dem[:n], inst.ex[:n],
                                           inst.cap, inst.x0r, inst.sl, inst.Sl, inst.X0, inst.s,
                                           inst.S)
        t0 = time.perf_counter()
        ow.seq_sim(cut(200), net)
        per_step = max((time.perf_counter() - t0) / 200, 1e-9)
        sub = cut(max(200, min(inst.T, int(budget / per_step))))
        for _ in range(max(0, args.warmup)):
            ow.seq_sim(sub, net)
        t0 = time.perf_counter()
        for _ in range(per):
            ow.seq_sim(sub, net)
        el = time.perf_counter() - t0
        value = per * sub.T / el
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": per, "warmup": args.warmup,
            "ms_per_step": 1000 * inst.T / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32+f32", "data": "synthetic",
            "config": owmr_config(args, inst, net, DEFAULT_MAX_STEPS["owmr_base"], inst.N),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {sub.T} of {inst.T} steps per step, sequential C "
                                       "oracle with the network, 1 thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    if args.workload == "batch_uneven":
        from paper_2406_01939_b300 import synth
        insts, pols = synth.batch_uneven(args.seed)
        rate, sample, _ = batch_oracle_sample(insts, pols, budget)
        total_T = sum(i.T for i in insts)
        t0 = time.perf_counter()
        n_orders = 0
        for _ in range(per):
            r, _, done = batch_oracle_sample(insts, pols, budget)
            n_orders += sum(insts[b].T for b, _ in done)
        el = time.perf_counter() - t0
        value = n_orders / el
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": per, "warmup": args.warmup, "ms_per_step": 1000 * total_T / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32",
            "data": "synthetic", "config": batch_config(args, insts, None),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: " + sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    inst, pol, _ = make_workload(args, args.seed)
    # each step: the full trajectory, or a prefix of it when a full run exceeds the budget
    probe = prefix_instance(inst, min(inst.T, 2048))
    t0 = time.perf_counter()
    oracle.seq_sim(probe, pol)
    per_order = max((time.perf_counter() - t0) / probe.T, 1e-9)
    Ts = inst.T if per_order * inst.T <= budget else max(probe.T, int(budget / per_order))
    sub = inst if Ts == inst.T else prefix_instance(inst, Ts)
    for _ in range(max(0, args.warmup)):
        oracle.seq_sim(sub, pol)
    t0 = time.perf_counter()
    for _ in range(per):
        oracle.seq_sim(sub, pol)
    el = time.perf_counter() - t0
    value = per * sub.T / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": per, "warmup": args.warmup, "ms_per_step": 1000 * el / per * inst.T / sub.T,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.workload == "mlp_medium" else "int32",
        "data": "synthetic",
        "config": dict(workload_config(args, inst),
                       parallelism=f"one trajectory per rank ({max(1, int(args.gpus))})"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": (f"full {inst.T}-order trajectory per step" if sub.T == inst.T else
                                    f"first {sub.T} of {inst.T} orders per step") +
                                   ", sequential C oracle, 1 thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def pass_trace_of(tr, iters):
    """Per-pass record (pic_sim_opts.trace rows) as lists: prefix and replay
    phase times, policy calls, work units, and the largest unit's calls and
    orders."""
    n = min(iters, tr.shape[0])
    ts, tr_end = tr[:n, 0], tr[:n, 1]
    prev = np.r_[0, tr_end[:-1]]
    return {"prefix_us": ((ts - prev) / 1e3).round(1).tolist(),
            "replay_us": ((tr_end - ts) / 1e3).round(1).tolist(),
            "policy_calls": tr[:n, 2].tolist(), "units": tr[:n, 3].tolist(),
            "longest_unit_calls": tr[:n, 4].tolist(), "longest_unit_orders": tr[:n, 5].tolist()}


def critical_path(trace, t_dec_us, kernel_ms, what):
    """A lower bound model of the persistent kernel's time from its pass trace:
    every pass waits for its largest work unit, whose policy calls run one after
    another (t_dec_us each, the measured latency of one decision by one warp),
    and costs at least the cheapest pass of the call (t_floor: the barriers and
    the prefix phase with almost no work).  frac = bound / kernel time."""
    if not trace or not trace["policy_calls"]:
        return None
    pass_us = [a + b for a, b in zip(trace["prefix_us"], trace["replay_us"])]
    floor_us = min(pass_us)
    chain = sum(trace["longest_unit_calls"])
    bound_us = chain * t_dec_us + floor_us * len(pass_us)
    return {"bound_us": bound_us, "kernel_us": kernel_ms * 1000.0,
            "frac": bound_us / (kernel_ms * 1000.0), "passes": len(pass_us),
            "sequential_decisions": int(chain), "t_decision_us": t_dec_us,
            "t_pass_floor_us": floor_us,
            "model": "sum over passes of (largest unit's policy calls x t_decision) + passes x "
                     "t_pass_floor; " + what}


def fp32_scored(res):
    """MLP decisions that ran the FP32 scorer: not taken from tensor-core tile
    scores and not from the saturated-state table (those cost no scorer FLOPs
    on the CUDA cores)."""
    return res["mlp_calls"] - res["tc_decisions"] - res["sat_decisions"]


def mlp_roofline(mlp_calls, N, ms, kernel):
    flops = mlp_calls * mlp_flops_per_call(N)
    achieved = flops / (ms / 1000.0) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None, "kernel": kernel,
            "peak_kind": "derived: 148 SMs x 128 FP32 lanes x 2 FLOP x 2.032 GHz",
            "algorithmic_flops": flops}


def sim_roofline(r, N, ms):
    """Roofline of a batch simulation launch (r: the result's counters).  With
    tensor-core waves: the rows whose scores the tensor cores produced (kept or
    re-scored as near ties) against the sustained BF16 peak (the launch runs
    inside a long step); with the warp kernel: the FP32-scored decisions
    against the FP32 ALU peak."""
    if r["wave"]:
        flops = (r["tc_decisions"] + r["rescored"]) * mlp_flops_per_call(N)
        peak, kind = load_bf16_peak(sustained=True)
        ach = flops / (ms / 1000.0) / 1e12
        return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": profiled_traffic("wave"),
                "kernel": "k_picard_wave (tcgen05 waves of 128 rows; all passes)",
                "peak_kind": kind + " BF16 dense", "algorithmic_flops": flops,
                "rows": "tensor-core rows kept or re-scored; table and FP32-scorer decisions "
                        "excluded"}
    roof = mlp_roofline(fp32_scored(r), N, ms,
                        "k_picard_batch (warp per work unit; all passes; MLP scorer FP32 FMA)")
    roof["traffic"] = profiled_traffic("batch")
    return roof


def run_batch(args, dev, world, rank):
    """Batch workload: every step simulates all trajectories of the batch in one
    persistent launch (CUDA graph)."""
    import torch
    import torch.distributed as dist
    import paper_2406_01939_b300 as pic
    from paper_2406_01939_b300 import synth
    from paper_2406_01939_b300.session import DeviceBatch

    insts, pols = synth.batch_uneven(rank_seed(args.seed, rank), **({"B": args.B} if args.B else {}))
    db = DeviceBatch(insts, device=dev)
    T = db.T
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    act = torch.empty(T, dtype=torch.int8, device=dev)
    flags = pic.PIC_FLAG_TIMING | pic.PIC_FLAG_GRAPH | args.flags

    def step():
        return db.simulate(pols, "picard", num_chunks=chunks_of(args), seg_window=args.seg_window,
                           flags=flags, want_stock=False, out=act)

    t_tune = time.perf_counter()
    first = step()  # runs the autotuner when chunks = 0
    t_tune = time.perf_counter() - t_tune
    for _ in range(max(3, args.warmup)):
        r = step()
    stream = torch.cuda.current_stream(dev)
    clocks = Clocks(int(str(dev).split(":")[-1]) if ":" in str(dev) else 0)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    evs, results = [], []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        results.append(step())
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    value, t_ms = job_rate(T, args.steps, sum(a.elapsed_time(b) for a, b in evs), world, dev)
    last = results[-1]
    sim_ms = statistics.median(r["sim_ms"] for r in results)
    # one extra (untimed) call with the per-pass trace, and the latency of one MLP
    # decision by one warp (the longest work units are MLP runs): the one-warp
    # sequential simulator on the first orders of the first MLP trajectory
    tr = np.zeros((4096, 6), np.int64)
    db.simulate(pols, "picard", num_chunks=last["num_chunks"], seg_window=last["seg_window"],
                flags=args.flags | (pic.PIC_FLAG_WAVE if last["wave"] else 0), want_stock=False,
                out=act, trace=tr)
    pass_trace = pass_trace_of(tr, last["iters"])
    from paper_2406_01939_b300.session import DeviceInstance
    bm = next(b for b, p in enumerate(pols) if p.kind != "greedy")
    Tp = min(insts[bm].T, 16384)
    dp = DeviceInstance(prefix_instance(insts[bm], Tp), device=dev)
    pact = torch.empty(Tp, dtype=torch.int8, device=dev)
    tds = [dp.simulate(pols[bm], "sequential", flags=pic.PIC_FLAG_TIMING, want_stock=False,
                       out=pact)["total_ms"] for _ in range(3)]
    dp.close()
    t_dec_us = 1000.0 * statistics.median(tds[1:]) / Tp
    cp = critical_path(pass_trace, t_dec_us, sim_ms,
                       f"every unit's calls charged as MLP decisions; t_decision: one-warp "
                       f"sequential simulator on the first {Tp} orders of trajectory {bm} (MLP)")

    seq_ms, bit_exact_gpu = None, None
    if args.seq_steps > 0:
        seq_act = torch.empty(T, dtype=torch.int8, device=dev)
        seq_ms = []
        for i in range(args.seq_steps + 1):
            rs = db.simulate(pols, "sequential", flags=pic.PIC_FLAG_TIMING, want_stock=False,
                             out=seq_act)
            if i:
                seq_ms.append(rs["total_ms"])
        seq_ms = statistics.median(seq_ms)
        bit_exact_gpu = bool(torch.equal(seq_act, act)) and all(
            a["total_cost"] == b["total_cost"] and a["lost"] == b["lost"]
            for a, b in zip(rs["traj"], last["traj"]))

    # end to end: every step loads the trajectories into the batch instance from
    # pinned host arrays (pic_batch_load: H2D, id shift and range checks inside
    # the call) and simulates them with host outputs; the instance is created once
    # before the timed steps; chunking fixed to the tuned choice
    e2e_t, h2d, d2h, bit_exact_e2e = [], 0, 0, None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).pin_memory().numpy()
        host = [synth.Instance(i.T, i.N, i.K, i.R, pin(i.prod), pin(i.reg), pin(i.x0), pin(i.cost),
                               None) for i in insts]
        h2d = sum(i.prod.nbytes + i.reg.nbytes + i.x0.nbytes + i.cost.nbytes for i in host)
        host_act = torch.empty(T, dtype=torch.int8).pin_memory().numpy()
        d2h = host_act.nbytes + 24 * len(insts)
        hb = DeviceBatch(host, device=dev, mem=pic.PIC_MEM_HOST)
        for i in range(args.e2e_steps + 1):
            flush.fill_(1)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            hb.load(host, mem=pic.PIC_MEM_HOST)
            hb.simulate(pols, "picard", num_chunks=last["num_chunks"], seg_window=last["seg_window"],
                        flags=args.flags | (pic.PIC_FLAG_WAVE if last["wave"] else 0),
                        want_stock=False, out=host_act, out_mem=pic.PIC_MEM_HOST)
            t1 = time.perf_counter()
            if i:
                e2e_t.append(t1 - t0)
        hb.close()
        bit_exact_e2e = bool(np.array_equal(host_act, act.cpu().numpy()))
    e2e_value = job_rate(T, 1, 1000.0 * statistics.median(e2e_t), world, dev)[0] if e2e_t else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32", "data": "synthetic",
        "config": batch_config(args, insts, last),
        "iters": last["iters"],
        "iters_per_trajectory": {"min": min(t["iters"] for t in last["traj"]),
                                 "max": max(t["iters"] for t in last["traj"])},
        "seq_gpu": {"value": T / (seq_ms / 1000.0), "unit": UNIT, "ms": seq_ms,
                    "what": "one warp per trajectory, all trajectories in one launch"}
        if seq_ms else None,
        "speedup_vs_seq_gpu": seq_ms / (t_ms / args.steps) if seq_ms else None,
        "bit_exact_vs_seq_gpu": bit_exact_gpu,
        "autotune_s": t_tune,
        "phases_ms": {"per_call_work": sim_ms, "step_device": t_ms / args.steps},
        "policy_calls": last["policy_calls"], "mlp_calls": last["mlp_calls"],
        "tc_decisions": last["tc_decisions"], "sat_decisions": last["sat_decisions"],
        "near_ties": last["near_ties"],
        "segment_replays": last["seg_replays"],
        "roofline": sim_roofline(last, insts[0].N, sim_ms),
        "critical_path": cp,
        "pass_trace": pass_trace,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "bit_exact": bit_exact_e2e,
                "what": "pic_create_batch from pinned host arrays + pic_simulate_batch with host "
                        "outputs + release, per step"},
        "gpu_launches": int(last["launches"]) * args.steps,
        "clocks": clk,
        "wall_s_timed_loop": wall,
    }
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        rate, sample, done = batch_oracle_sample(insts, pols, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": sample}
        a = act.cpu().numpy()
        same = True
        for b, out in done:
            same &= bool(np.array_equal(out["actions"], a[db.offsets[b]:db.offsets[b + 1]]))
            same &= out["total_cost"] == last["traj"][b]["total_cost"]
        line["bit_exact_vs_oracle"] = same
        line["oracle_trajectories_checked"] = len(done)
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    db.close()


def grad_flops_per_order(N):
    """Algorithmic FLOPs of the gradient per order: hidden layer (stock rows),
    scores, dW2, W2 ds and dW1 (stock rows): five N x 256 products, 2 FLOP per
    FMA (the tensor-core kernel's split products and recomputation are extra)."""
    return 2 * 5 * N * 256


def run_pg(args, dev, world, rank):
    """Policy-gradient step: simulate the batch (Picard) with BF16(master), then
    the objective and gradient along those paths."""
    import torch
    import torch.distributed as dist
    import paper_2406_01939_b300 as pic
    from paper_2406_01939_b300 import synth
    from paper_2406_01939_b300.reinforce import Reinforce, flat_from_mlp
    from paper_2406_01939_b300.session import DeviceBatch

    B = args.B or 64
    insts, mlp = synth.pg_large(rank_seed(args.seed, rank), B=B)
    db = DeviceBatch(insts, device=dev)
    T, N = db.T, insts[0].N
    rf = Reinforce(db, ["gumbel"] * B, [1000 + b for b in range(B)], list(range(B)), insts[0].R,
                   num_chunks=chunks_of(args), seg_window=args.seg_window,
                   flags=pic.PIC_FLAG_TIMING | args.flags)
    master = flat_from_mlp(mlp, device=dev)
    acts = torch.empty(T, dtype=torch.int8, device=dev)
    grad = torch.empty_like(master)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        # one call: simulate the paths (Picard), then J and the gradient (tile kernel)
        e0 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        J, res = rf.step(master, grad, actions_out=acts)
        if world > 1:  # each rank holds its own trajectories: the batch's gradient and J
            from paper_2406_01939_b300.shard import gradient_all_reduce
            _, J = gradient_all_reduce(grad, J, device=dev)
        e2.record(stream)
        return J, res, (e0, e2)

    for _ in range(max(3, args.warmup)):
        step()
    clocks = Clocks(int(str(dev).split(":")[-1]) if ":" in str(dev) else 0)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    recs = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        recs.append(step())
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    value, t_ms = job_rate(T, args.steps, sum(a.elapsed_time(b) for _, _, (a, b) in recs), world, dev)
    J, res, _ = recs[-1]
    # the gradient kernel alone, timed separately along the last step's paths
    gts = []
    for _ in range(3):
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        rf.gradient(master, acts, grad)
        g1.record(stream)
        torch.cuda.synchronize(dev)
        gts.append(g0.elapsed_time(g1))
    bwd_ms = statistics.median(gts)
    # the sequential GPU simulator on the same batch (one warp per trajectory,
    # every trajectory in one launch, the same BF16 parameters and noise)
    from paper_2406_01939_b300.synth import Policy
    spols = [Policy("gumbel", mlp=mlp, seed=1000 + b, traj=b) for b in range(B)]
    seq_ms, bit_exact_gpu = None, None
    if args.seq_steps > 0:
        seq_act = torch.empty(T, dtype=torch.int8, device=dev)
        sms = [db.simulate(spols, "sequential", flags=pic.PIC_FLAG_TIMING, want_stock=False,
                           out=seq_act)["total_ms"] for _ in range(min(2, args.seq_steps) + 1)]
        seq_ms = statistics.median(sms[1:])
        bit_exact_gpu = bool(torch.equal(seq_act, acts))
    # end to end: every step loads the trajectories into the batch instance from
    # pinned host arrays (pic_batch_load), copies the master parameters from pinned
    # host memory, takes one gradient step and reads J back (a double); the
    # instance is created once before the timed steps
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).pin_memory().numpy()
        host = [synth.Instance(i.T, i.N, i.K, i.R, pin(i.prod), pin(i.reg), pin(i.x0), pin(i.cost),
                               None) for i in insts]
        master_h = master.cpu().pin_memory()
        h2d = sum(i.prod.nbytes + i.reg.nbytes + i.x0.nbytes + i.cost.nbytes for i in host) + \
            master_h.numel() * 4
        ts = []
        hb = DeviceBatch(host, device=dev, mem=pic.PIC_MEM_HOST)
        hrf = Reinforce(hb, ["gumbel"] * B, [1000 + b for b in range(B)], list(range(B)),
                        insts[0].R, num_chunks=res.num_chunks, seg_window=res.seg_window,
                        flags=args.flags | (pic.PIC_FLAG_WAVE if res.wave else 0))
        for i in range(min(3, args.e2e_steps) + 1):
            flush.fill_(1)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            hb.load(host, mem=pic.PIC_MEM_HOST)
            m_dev = master_h.to(dev, non_blocking=True)
            Jh, _ = hrf.step(m_dev, grad)
            t1 = time.perf_counter()
            if i:
                ts.append(t1 - t0)
        hb.close()
        e2e = {"value": job_rate(T, 1, 1000.0 * statistics.median(ts), world, dev)[0], "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 8,
               "objective_rel_diff": abs(Jh - J) / max(abs(J), 1e-300),
               "what": "pic_batch_load from pinned host arrays + master parameters H2D + "
                       "pic_policy_grad (simulate + J + gradient) with J returned to the host; "
                       "the batch instance created once before the timed steps"}
    flops = T * grad_flops_per_order(N)
    achieved = flops / (bwd_ms / 1000.0) / 1e12
    tc = not (args.flags & pic.PIC_FLAG_NO_TC)
    bf16_peak, bf16_kind = load_bf16_peak()
    # the dominant kernel is the simulation (all passes in one persistent launch)
    sim_roof = sim_roofline({"wave": res.wave, "mlp_calls": res.mlp_calls,
                             "tc_decisions": res.tc_decisions, "rescored": res.rescored,
                             "sat_decisions": res.sat_decisions}, N, res.sim_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32", "data": "synthetic",
        "config": {"workload": "pg_large",
                   "desc": (f"policy-gradient step, B={B} trajectories x T=2^20 orders, N={N}, "
                            f"K={insts[0].K}, R={insts[0].R}, Gumbel-max MLP policy, "
                            "BF16(master) parameters; Picard simulation + REINFORCE gradient"),
                   "B": B, "T_total": T, "N": N, "K": insts[0].K, "R": insts[0].R,
                   "chunks_per_trajectory": res.num_chunks, "seg_window": res.seg_window,
                   "l2": "inputs exceed L2; flushed between timed steps (256 MiB write)"},
        "iters": res.iters, "objective": J,
        "phases_ms": {"step": t_ms / args.steps, "simulation": res.sim_ms,
                      "gradient_call_on_given_paths": bwd_ms},
        "seq_gpu": {"value": T / (seq_ms / 1000.0), "unit": UNIT, "ms": seq_ms,
                    "what": "one warp per trajectory, all trajectories in one launch"}
        if seq_ms else None,
        "speedup_vs_seq_gpu": seq_ms / res.sim_ms if seq_ms else None,
        "speedup_basis": "sequential simulation / Picard simulation inside the step",
        "bit_exact_vs_seq_gpu": bit_exact_gpu,
        "policy_calls": res.policy_calls, "tc_decisions": res.tc_decisions,
        "sat_decisions": res.sat_decisions, "rescored": res.rescored,
        "near_ties": res.near_ties,
        "roofline": sim_roof,
        "roofline_gradient": ({"bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                      "frac": achieved / bf16_peak, "traffic": profiled_traffic("pg"),
                      "kernel": "k_pg_tc (tcgen05, BF16 split products, FP32 accumulation in TMEM)",
                      "peak_kind": bf16_kind + " BF16 dense (burst: the gradient call timed alone)",
                      "algorithmic_flops": flops} if tc else
                     {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                      "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                      "kernel": "k_pg_grad (FP32 CUDA cores)",
                      "peak_kind": "derived: 148 SMs x 128 FP32 lanes x 2 FLOP x 2.032 GHz",
                      "algorithmic_flops": flops}),
        "e2e": e2e,
        "gpu_launches": int(res.launches) * args.steps,
        "clocks": clk,
        "wall_s_timed_loop": wall,
        "cpu_baseline": None,
    }
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        rate, sample, out, covered = cpu_oracle_rate(insts[0], spols[0], args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "trajectory 0: " + sample}
        line["bit_exact_vs_oracle"] = bool(np.array_equal(out["actions"],
                                                          acts[:covered].cpu().numpy()))
        line["oracle_orders_checked"] = covered
    if rank == 0:
        print(json.dumps(line), flush=True)
    db.close()


def owmr_flops_per_call(H):
    """FLOPs of one retailer-network call: 3H + H^2 + H FMA, 2 FLOP each."""
    return 2 * (3 * H + H * H + H)


def owmr_config(args, inst, net, W, P):
    return {"workload": "owmr_base",
            "desc": (f"OWMR inventory control (App. B.3 base case): T={inst.T} unit demands over "
                     f"N={inst.N} stores ({'uniform' if not args.skew else f'weights (1-{args.skew})^n'}), "
                     "stores (s_n,S_n)=(10,20) capacity 24, central "
                     f"(s,S)=({inst.s},{inst.S}), retailer network 3-{net.H}-{net.H}-1 BF16 "
                     "N(0,0.02) fed (stock, demand, steps since the store's previous demand/4096)"),
            "T": inst.T, "N": inst.N, "hidden": net.H, "procs": P, "max_steps": W, "skew": args.skew,
            "l2": "working set (about 0.3 GB) exceeds L2; flushed between timed steps (256 MiB write)"}


def run_owmr(args, dev, world, rank):
    """OWMR (Appendix B): one Picard simulation per step, from the demand stream
    resident in HBM (per-processor step tables, every pass to the fixed point,
    actions and final state)."""
    import torch
    import paper_2406_01939_b300 as pic
    from paper_2406_01939_b300 import synth
    from paper_2406_01939_b300.owmr import (DeviceOwmr, DeviceOwmrNet, pic_owmr_create,
                                            pic_owmr_desc, pic_owmr_destroy, pic_owmr_opts,
                                            pic_owmr_policy, pic_owmr_simulate)
    inst, net = synth.owmr_base(rank_seed(args.seed, rank), a=args.skew,
                                **({"T": args.T} if args.T else {}))
    W = args.max_steps if args.max_steps >= 0 else DEFAULT_MAX_STEPS["owmr_base"]
    P = inst.N
    d = DeviceOwmr(inst, device=dev)
    dn = DeviceOwmrNet(net, device=dev)
    T = inst.T
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    step = lambda: d.simulate(dn, num_procs=P, max_steps=W, timing=True, flags=args.flags)
    for _ in range(max(3, args.warmup)):
        r = step()
    clocks = Clocks(int(str(dev).split(":")[-1]) if ":" in str(dev) else 0)
    torch.cuda.synchronize(dev)
    evs, results = [], []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        results.append(step())
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    value, t_ms = job_rate(T, args.steps, sum(a.elapsed_time(b) for a, b in evs), world, dev)
    last = results[-1]
    act = last["actions"].clone()
    state = last["state"].clone()

    # the sequential GPU simulator on a prefix (a prefix of the path depends only
    # on the prefix of the demand stream); its rate is the speedup denominator
    seq = None
    if args.seq_steps > 0:
        Tp = min(T, 200_000)
        pre = synth.OwmrInstance(Tp, inst.N, inst.ret[:Tp], inst.dem[:Tp], inst.ex[:Tp], inst.cap,
                                 inst.x0r, inst.sl, inst.Sl, inst.X0, inst.s, inst.S)
        dp = DeviceOwmr(pre, device=dev)
        sr = dp.simulate(dn, mode="sequential", timing=True)
        rate = Tp / (sr["ms"] / 1000.0)
        seq = {"value": rate, "unit": UNIT, "ms_prefix": sr["ms"], "prefix_steps": Tp,
               "ms_full_horizon_est": 1000.0 * T / rate,
               "bit_exact_on_prefix": bool(torch.equal(sr["actions"], act[:Tp]))}
        dp.close()

    # end to end through host buffers: create from pinned host arrays, simulate
    # with host outputs, release
    pin = lambda a: torch.from_numpy(np.array(a, dtype=np.int32, copy=True)).pin_memory()
    host = [pin(getattr(inst, k)) for k in ("ret", "dem", "ex", "cap", "x0r", "sl", "Sl")]
    host_act = torch.empty(T, dtype=torch.int32).pin_memory()
    host_state = torch.empty(inst.N + 1, dtype=torch.int32).pin_memory()
    h2d = sum(x.numel() * 4 for x in host)
    d2h = (T + inst.N + 1) * 4
    e2e_t = []
    for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        desc = pic_owmr_desc(T, inst.N, *[x.data_ptr() for x in host], inst.X0, inst.s, inst.S,
                             pic.PIC_MEM_HOST, None)
        h = pic_owmr_create(desc)
        opts = pic_owmr_opts(pic.PIC_MODE_PICARD, P, 0, 0, None, 0, W)
        st, res = pic_owmr_simulate(h, dn.policy(), opts, host_act, host_state, pic.PIC_MEM_HOST)
        pic_owmr_destroy(h)
        t1 = time.perf_counter()
        if st != pic.PIC_OK:
            raise RuntimeError(f"e2e simulate failed: {st}")
        if i >= 1:
            e2e_t.append(t1 - t0)
    e2e_value = T / statistics.median(e2e_t) if e2e_t else None
    bit_exact_e2e = bool(torch.equal(host_act, act.cpu())) if e2e_t else None

    sim_ms = statistics.median(r["ms"] for r in results)
    flops = last["policy_calls"] * owmr_flops_per_call(net.H)
    achieved = flops / (sim_ms / 1000.0) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32", "data": "synthetic",
        "config": owmr_config(args, inst, net, W, P),
        "iters": last["iters"], "replenishments": last["R"],
        "passes_bound_2R_plus_2": 2 * last["R"] + 2,
        "policy_calls": last["policy_calls"], "eval_rounds": last["eval_rounds"],
        "seq_gpu": seq,
        "speedup_vs_seq_gpu": (seq["ms_full_horizon_est"] / (t_ms / args.steps)) if seq else None,
        "phases_ms": {"call": sim_ms, "step_device": t_ms / args.steps},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": profiled_traffic("owmr"),
                     "kernel": "k_owmr_picard (persistent, all passes; FP32 network rounds)",
                     "peak_kind": "derived: 148 SMs x 128 FP32 lanes x 2 FLOP x 2.032 GHz",
                     "algorithmic_flops": flops},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "bit_exact": bit_exact_e2e,
                "what": "pic_owmr_create from pinned host arrays + pic_owmr_simulate with host "
                        "outputs + pic_owmr_destroy, per step"},
        "gpu_launches": int(last["launches"]) * args.steps,
        "clocks": clk,
        "wall_s_timed_loop": wall,
    }
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        from oracle import owmr as ow
        Tc, el, out = 1000, 0.0, None
        while True:
            pre = synth.OwmrInstance(Tc, inst.N, inst.ret[:Tc], inst.dem[:Tc], inst.ex[:Tc],
                                     inst.cap, inst.x0r, inst.sl, inst.Sl, inst.X0, inst.s, inst.S)
            t0 = time.perf_counter()
            out = ow.seq_sim(pre, net)
            el = time.perf_counter() - t0
            if el * 4 > args.cpu_seconds or Tc >= T:
                break
            Tc = min(T, Tc * 4)
        line["cpu_baseline"] = {"value": Tc / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {Tc} of {T} steps, sequential C oracle with the "
                                          f"width-{net.H} network, 1 thread ({el:.1f} s)"}
        line["bit_exact_vs_oracle"] = bool(np.array_equal(out["actions"], act.cpu().numpy()[:Tc]))
        line["oracle_steps_checked"] = Tc
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    d.close()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    import torch
    import torch.distributed as dist
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    if args.workload in ("batch_uneven", "pg_large", "owmr_base"):
        {"batch_uneven": run_batch, "pg_large": run_pg, "owmr_base": run_owmr}[args.workload](
            args, dev, world, rank)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    if args.chunk_sweep:
        for M in [int(x) for x in args.chunk_sweep.split(",") if x.strip()]:
            args.chunks = M
            run_single(args, dev, world, rank)
    else:
        run_single(args, dev, world, rank)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_single(args, dev, world, rank):
    """Single-trajectory FO workloads: one whole simulation per step."""
    import torch
    import torch.distributed as dist
    import paper_2406_01939_b300 as pic
    from paper_2406_01939_b300 import synth as synth_mod
    from paper_2406_01939_b300.session import DeviceInstance, DevicePolicy

    sharded = args.shard == "products"
    if sharded and (getattr(args, "partition", "chunks") != "chunks" or args.workload == "capacity_large"):
        raise SystemExit("--shard products: contiguous chunks, no node capacity")
    # sharded: every rank builds the same trajectory and keeps its products' orders
    inst, hpol, _ = make_workload(args, args.seed if sharded else rank_seed(args.seed, rank))
    T_job = inst.T
    if sharded:
        from paper_2406_01939_b300 import shard as shard_mod
        owner = shard_mod.product_shards(inst.prod, inst.K, world)
        inst, shard_times, _ = shard_mod.shard_instance(inst, owner, rank)
    di = DeviceInstance(inst, device=dev)
    pol = DevicePolicy(hpol, dev)
    T = inst.T
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    max_steps = args.max_steps if args.max_steps >= 0 else DEFAULT_MAX_STEPS.get(args.workload, 0)
    if not args.seg_window:
        args.seg_window = DEFAULT_SEG_WINDOW.get(args.workload, 0)

    products = args.partition == "products"
    rand = args.partition == "random"
    if (products or rand) and (args.workload == "mlp_medium" or max_steps):
        raise SystemExit("--partition products/random: greedy / bid-price workloads, no max_steps")
    fo_mode = {"chunks": "picard", "products": "products", "random": "assigned"}[args.partition]
    fo_chunks = 0 if products else chunks_of(args)
    proc_host = synth_mod.uniform_assignment(T, fo_chunks, seed=args.seed) if rand else None
    proc_dev = torch.as_tensor(proc_host).to(dev) if rand else None

    # contiguous chunks: the order tables (stable sort by product, runs, segments,
    # longest-first order) depend only on the order stream and the chunking, so
    # the timed steps keep them on the instance (PIC_FLAG_REUSE_TABLES), as in
    # policy evaluation over a fixed demand stream; the same steps with the
    # tables rebuilt every call are timed too (fresh_tables), and the e2e path
    # reloads the inputs, which always rebuilds them
    reuse = pic.PIC_FLAG_REUSE_TABLES if args.partition == "chunks" and not args.fresh_tables else 0

    def step(out, extra=reuse):
        r = di.simulate(pol, fo_mode, num_chunks=fo_chunks, seg_window=args.seg_window,
                        proc=proc_dev,
                        flags=pic.PIC_FLAG_TIMING | args.flags | extra, want_stock=False, out=out,
                        max_steps=max_steps)
        if sharded and world > 1:  # the trajectory's totals: one all-reduce per step
            r["total_cost"], r["lost"], r["iters"] = shard_mod.join_scalars(
                r["total_cost"], r["lost"], r["iters"], device=dev)
        return r

    act = torch.empty(T, dtype=torch.int8, device=dev)
    for _ in range(max(3, args.warmup)):
        r = step(act)
    stream = torch.cuda.current_stream(dev)
    clocks = Clocks(dev.index or 0)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    evs = []
    results = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)  # evict the previous step's working set from L2 (untimed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        results.append(step(act))
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    value, t_ms = job_rate(T, args.steps, sum(step_ms), world, dev)  # sharded: sum of T = T_job
    last = results[-1]
    fresh = None
    if reuse:  # the same steps with the tables rebuilt on every call (untimed for value)
        fms, fprep = [], []
        for _ in range(min(args.steps, 10)):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rf = step(act, extra=0)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            fms.append(e0.elapsed_time(e1))
            fprep.append(rf["prep_ms"])
        fresh = {"ms_per_step": statistics.median(fms), "tables_ms": statistics.median(fprep),
                 "orders_per_s": T / (statistics.median(fms) / 1000.0),
                 "what": "the same step with the order tables rebuilt on every call"}
    # one extra (untimed) call with the per-pass trace (contiguous chunks)
    pass_trace = None
    if args.partition == "chunks":
        tr = np.zeros((4096, 6), np.int64)
        di.simulate(pol, "picard", num_chunks=chunks_of(args), seg_window=args.seg_window,
                    flags=args.flags, want_stock=False, out=act, trace=tr, max_steps=max_steps)
        pass_trace = pass_trace_of(tr, last["iters"])
    sim_ms = statistics.median(r["sim_ms"] for r in results)
    prep_ms = statistics.median(r["prep_ms"] for r in results)
    iters = last["iters"]

    # sequential GPU simulator (the speedup denominator), same instance
    seq_ms, bit_exact_gpu = None, None
    if args.seq_steps > 0:
        seq_act = torch.empty(T, dtype=torch.int8, device=dev)
        seq_ms = []
        # the MLP's fastest sequential simulator shares each decision between four warps
        seq_flags = pic.PIC_FLAG_TIMING | (pic.PIC_FLAG_WARP_GROUP if args.workload == "mlp_medium"
                                           else 0)
        for i in range(args.seq_steps + 1):
            r = di.simulate(pol, "sequential", flags=seq_flags, want_stock=False, out=seq_act)
            if i:
                seq_ms.append(r["total_ms"])
            seq_res = r
        seq_ms = statistics.median(seq_ms)
        bit_exact_gpu = bool(torch.equal(seq_act, act)) and seq_res["total_cost"] == last["total_cost"]
    # latency of one decision by one warp (the Picard kernel's unit of sequential
    # work): the one-warp sequential simulator on the first orders of the trajectory
    t_dec_us = None
    if args.partition == "chunks":
        Tp = min(T, 16384)
        dp = DeviceInstance(prefix_instance(inst, Tp), device=dev)
        pact = torch.empty(Tp, dtype=torch.int8, device=dev)
        tds = [dp.simulate(pol, "sequential", flags=pic.PIC_FLAG_TIMING, want_stock=False,
                           out=pact)["total_ms"] for _ in range(3)]
        t_dec_us = 1000.0 * statistics.median(tds[1:]) / Tp
        dp.close()

    # end to end through host buffers: H2D of the inputs, simulate, D2H of the actions
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).pin_memory()
    host = {k: pin(getattr(inst, k)) for k in ("prod", "reg", "x0", "cost")}
    host["lam"] = pin(inst.lam) if inst.lam is not None else None
    host["cap"] = pin(inst.cap) if getattr(inst, "cap", None) is not None else None
    proc_pin = pin(proc_host) if rand else None
    proc_e2e = torch.empty(T, dtype=torch.int32, device=dev) if rand else None
    host_np = {k: (v.numpy() if v is not None else None) for k, v in host.items()}
    host_act = torch.empty(T, dtype=torch.int8).pin_memory().numpy()
    opts = pic.make_opts(fo_mode, fo_chunks, out_mem=pic.PIC_MEM_HOST, seg_window=args.seg_window,
                         proc=proc_e2e,
                         flags=args.flags, max_steps=max_steps)
    h2d = sum(v.nbytes for v in host_np.values() if v is not None) + (proc_host.nbytes if rand else 0)
    d2h = host_act.nbytes + 64  # actions + the result record
    e2e_t = []
    for i in range(args.e2e_steps + 2 if args.e2e_steps > 0 else 0):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        di.load_host(host_np)
        if rand:
            proc_e2e.copy_(proc_pin, non_blocking=True)  # the assignment is an input too
        st, res = pic.pic_simulate(di.handle, pol.struct, opts, host_act)
        t1 = time.perf_counter()
        if i >= 2:
            e2e_t.append(t1 - t0)
    e2e_value = job_rate(T, 1, 1000.0 * statistics.median(e2e_t), world, dev)[0] if e2e_t else None
    bit_exact_e2e = bool(np.array_equal(host_act, act.cpu().numpy())) if e2e_t else None

    # roofline of the dominant kernel (the persistent Picard kernel)
    N = inst.N
    if products or rand:
        # per pass and order: its time, product, region, cached action (read and
        # written) and, with capacity, its cached success (4 + 4 + 4 + 2 (+ 4) B), and
        # its cost row (N x 4 B).  Products: the pass is bound by the longest
        # product's chain of orders, walked one at a time by one warp; random: by the
        # start latency of the ~10^5-10^6 (product, process) chains.  The fraction is
        # low by design.
        per = 14 + 4 * N + (4 if getattr(inst, "cap", None) is not None else 0)
        alg_bytes = last["policy_calls"] * per
        acap = rand and getattr(inst, "cap", None) is not None
        if acap:
            # every process replays the horizon up to its last own order: per
            # order-step its product, owner and cached action (4 + 4 + 1 B); per own
            # order its region, cost and lambda rows and the new action (5 + 8 N B)
            lastm = np.full(int(proc_host.max()) + 1, -1, np.int64)
            np.maximum.at(lastm, proc_host.astype(np.int64), np.arange(T, dtype=np.int64))
            walk = int((lastm + 1).sum())
            alg_bytes = last["iters"] * walk * 9 + last["policy_calls"] * (5 + 8 * N)
        achieved = alg_bytes / (sim_ms / 1000.0) / 1e9
        peak, peak_kind = load_peaks()
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": ("k_part_walk plus the per-pass sorts (all passes)" if products else
                               "k_acap_pass (every process replays its view; all passes)"
                               if getattr(inst, "cap", None) is not None else
                               "k_assign_walk plus the per-pass sorts (all passes)"),
                    "peak_kind": peak_kind, "algorithmic_bytes": alg_bytes,
                    "critical_path_orders_per_pass": int(np.bincount(inst.prod).max()) if products
                    else int(lastm.max() + 1) if acap
                    else int(np.unique(proc_host.astype(np.int64) * inst.K + inst.prod,
                                       return_counts=True)[1].max())}
    elif args.workload == "mlp_medium":
        roofline = mlp_roofline(fp32_scored(last), N, sim_ms, "k_picard_mlp (persistent, all passes)")
        roofline["traffic"] = profiled_traffic("mlp")
    elif args.workload == "capacity_large":
        # the method's bytes: per replayed order its record (product and region,
        # 2 B each), its sorted position (4 B) and its cached action read and
        # written (1 B each); per replayed run the x0 row and the lambda row of its
        # product (N x 4 B each).  The kernel's own histogram and prefix rows are
        # intermediates, not counted (they show in the measured traffic).
        alg_bytes = last["policy_calls"] * 10 + last["seg_replays"] * 8 * N
        achieved = alg_bytes / (sim_ms / 1000.0) / 1e9
        peak, peak_kind = load_peaks()
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": profiled_traffic("capacity"),
                    "kernel": "k_picard_cap (persistent, all passes)", "peak_kind": peak_kind,
                    "algorithmic_bytes": alg_bytes}
    else:
        # the method's bytes (as above): 10 B per replayed order, and the x0 and
        # lambda rows (N x 4 B each) per replayed work unit of one product
        alg_bytes = last["policy_calls"] * 10 + last["seg_replays"] * 8 * N
        achieved = alg_bytes / (sim_ms / 1000.0) / 1e9
        peak, peak_kind = load_peaks()
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": profiled_traffic(),
                    "kernel": "k_picard_int (persistent, all passes)", "peak_kind": peak_kind,
                    "algorithmic_bytes": alg_bytes}

    cp = critical_path(pass_trace, t_dec_us, sim_ms,
                       "t_decision: one-warp sequential simulator on the first "
                       f"{min(T, 16384)} orders") if t_dec_us else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "vs_baseline": None,
        "dtype": "f32" if args.workload == "mlp_medium" else "int32", "data": "synthetic",
        "config": dict(workload_config(args, inst),
                       **({"T": T_job, "parallelism": f"products of one trajectory over {world} "
                           "ranks (balanced by demand); cost, lost and passes all-reduced each step"}
                          if sharded else {"parallelism": f"one trajectory per rank ({world})"})),
        "iters": iters,
        "seq_gpu": {"value": T / (seq_ms / 1000.0), "unit": UNIT, "ms": seq_ms} if seq_ms else None,
        "speedup_vs_seq_gpu": seq_ms / (t_ms / args.steps) if seq_ms else None,
        "bit_exact_vs_seq_gpu": bit_exact_gpu,
        "phases_ms": {"tables": prep_ms, "picard_kernel": sim_ms,
                      "step_device": t_ms / args.steps},
        "order_tables": ("kept on the instance across steps (PIC_FLAG_REUSE_TABLES; built by the "
                         "warm-up calls)" if reuse else "rebuilt on every call"),
        "fresh_tables": fresh,
        "speedup_vs_seq_gpu_fresh_tables": (seq_ms / fresh["ms_per_step"]) if (fresh and seq_ms) else None,
        "policy_calls": last["policy_calls"], "segment_replays": last["seg_replays"],
        "mlp_calls": last["mlp_calls"], "tc_decisions": last["tc_decisions"],
        "sat_decisions": last["sat_decisions"], "near_ties": last["near_ties"],
        "pass_trace": pass_trace,
        "roofline": roofline,
        "critical_path": cp,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "bit_exact": bit_exact_e2e},
        "gpu_launches": int(last["launches"]) * args.steps,
        "clocks": clk,
        "wall_s_timed_loop": wall,
    }
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        rate, sample, out, covered = cpu_oracle_rate(inst, hpol, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": sample}
        same = bool(np.array_equal(out["actions"], act.cpu().numpy()[:covered]))
        if covered == T:
            same = same and out["total_cost"] == last["total_cost"]
        line["bit_exact_vs_oracle"] = same
        line["oracle_orders_checked"] = covered
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    di.close()


if __name__ == "__main__":
    main()
