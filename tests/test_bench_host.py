"""Host-side arithmetic of bench.py (no GPU): the per-pass trace record, the
critical-path model, the rooflines of the batch and policy-gradient lines, the
peak loader and the source-hash check that lets a committed profile supply a
kernel's DRAM traffic only while the kernel's source is unchanged."""
import json
import os

import numpy as np
import pytest

import bench


def test_pass_trace_of_splits_phases():
    tr = np.zeros((8, 6), np.int64)
    # end of phase S and end of phase R per pass (ns since the launch), calls,
    # units, the largest unit's calls and orders
    tr[0] = [1000, 5000, 10, 3, 4, 6]
    tr[1] = [7000, 9000, 2, 1, 2, 2]
    t = bench.pass_trace_of(tr, 2)
    assert t["prefix_us"] == [1.0, 2.0]
    assert t["replay_us"] == [4.0, 2.0]
    assert t["policy_calls"] == [10, 2] and t["units"] == [3, 1]
    assert t["longest_unit_calls"] == [4, 2] and t["longest_unit_orders"] == [6, 2]


def test_critical_path_model():
    trace = {"prefix_us": [1.0, 2.0, 1.0], "replay_us": [9.0, 4.0, 2.0],
             "policy_calls": [100, 10, 1], "longest_unit_calls": [10, 4, 1]}
    cp = bench.critical_path(trace, 0.5, 0.05, "test")
    # 15 decisions x 0.5 us + 3 passes x the cheapest pass (3 us)
    assert cp["bound_us"] == pytest.approx(15 * 0.5 + 3 * 3.0)
    assert cp["frac"] == pytest.approx(cp["bound_us"] / 50.0)
    assert cp["sequential_decisions"] == 15 and cp["passes"] == 3
    assert bench.critical_path(None, 0.5, 1.0, "") is None
    assert bench.critical_path(dict(trace, policy_calls=[]), 0.5, 1.0, "") is None


def test_sim_roofline_branches(monkeypatch):
    monkeypatch.setattr(bench, "profiled_traffic", lambda kind: {"wave": 7.0, "batch": 9.0}[kind])
    r = {"wave": True, "tc_decisions": 1000, "rescored": 24, "mlp_calls": 5000, "sat_decisions": 100}
    roof = bench.sim_roofline(r, 64, 2.0)
    flops = 1024 * bench.mlp_flops_per_call(64)
    peak, _ = bench.load_bf16_peak(sustained=True)
    assert roof["bound"] == "tensor" and roof["algorithmic_flops"] == flops
    assert roof["achieved"] == pytest.approx(flops / 2e-3 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / peak) and roof["traffic"] == 7.0
    roof = bench.sim_roofline(dict(r, wave=False), 64, 2.0)
    assert roof["bound"] == "alu" and roof["traffic"] == 9.0
    # FP32-scored decisions only: tile and table decisions take no scorer FLOPs
    assert roof["algorithmic_flops"] == (5000 - 1000 - 100) * bench.mlp_flops_per_call(64)


def test_bf16_peak_burst_and_sustained(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_bf16_peak() == (1800.0, "fallback")
    assert bench.load_bf16_peak(sustained=True)[0] == 1400.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps(
        {"hbm_gbs": 6000.0, "bf16_tflops": 1700.0, "bf16_tflops_sustained": 1300.0}))
    assert bench.load_bf16_peak() == (1700.0, "measured")
    assert bench.load_bf16_peak(sustained=True)[0] == 1300.0
    assert bench.load_peaks() == (6000.0, "measured")


def test_profiled_traffic_requires_the_profiled_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2406_01939_b300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    files = bench._KERNEL_FILES["int"]
    for f in files:
        (csrc / f).write_text(f"// {f}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash("int")
    prof = tmp_path / "profiles" / bench._PROFILES["int"]
    prof.write_text(f"summary\nkernel_source_hash: {h}\ndram_bytes_per_launch: 12345\n")
    assert bench.profiled_traffic("int") == 12345.0
    (csrc / files[0]).write_text("// edited\n")  # the kernel changed since the capture
    assert bench.profiled_traffic("int") is None
    os.remove(prof)
    assert bench.profiled_traffic("int") is None


def test_committed_profiles_name_their_kernels():
    """Every profile the bench may read exists, carries a source hash, and gives
    the command that produced it."""
    for kind, name in bench._PROFILES.items():
        text = open(os.path.join(bench.ROOT, "profiles", name)).read()
        assert "kernel_source_hash:" in text, name
        assert "ncu " in text and "--clock-control none" in text, name
