"""bench.py's bookkeeping on CPU: the issue-slot roofline arithmetic, the
workload overrides, that the committed DRAM-traffic record belongs to the
kernel source as it is now (the bench reports traffic only then), and the
reference arm's line (the oracle timed on the host cores)."""
import argparse
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_alu_roofline_arithmetic():
    r = bench.alu_roofline(150e9, "accurate", 2000.0)
    peak = 152 * 4 * 32 * 2000e6 / 1e12                 # T thread-instructions/s
    assert r["bound"] == "alu" and r["unit"] == "Tinstr/s"
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(bench.ALG_INSTR_PER_UPDATE["accurate"] * 150e9 / 1e12)
    assert r["frac"] == pytest.approx(bench.ALG_INSTR_PER_UPDATE["accurate"] * 150e9 / 1e12 / peak)
    assert bench.alu_roofline(150e9, "fast", 2000.0)["frac"] < r["frac"]


def test_workload_overrides():
    a = argparse.Namespace(workload="large", sweeps=None, side=None)
    w = bench.workload(a)
    assert (w.L, w.sweeps, w.beta, w.seed) == (4096, 1000, 1.12, 7)
    a = argparse.Namespace(workload="large", sweeps=5, side=2048)
    w = bench.workload(a)
    assert (w.L, w.sweeps) == (2048, 5) and "L2048" in w.name and w.updates == 2048 * 2048 * 5
    w = bench.workload(argparse.Namespace(workload="huge", sweeps=None, side=None))
    assert (w.L, w.sweeps) == (16384, 200)


def test_traffic_record_matches_the_kernel_source():
    """profiles/traffic.json must have been taken from the kernel source as
    committed: re-capture it (ncu, the command it records) after any change
    to the files its hash covers."""
    from paper_0811_2111_gb300 import build as B
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    assert d["source_hash"] == B.source_hash(), "traffic.json is stale"
    assert d["dram_bytes_per_launch"] == d["dram_bytes_read_per_launch"] + d["dram_bytes_write_per_launch"]
    assert bench.profiled_traffic() == d["dram_bytes_per_launch"]
    # about the algorithmic 8 B per update of the bench step it records
    assert 0.5 < d["dram_bytes_per_launch"] / d["algorithmic_bytes_per_launch"] < 1.5


def test_reference_arm_line():
    """`bench.py --impl reference` times the oracle on the host cores (no GPU
    needed) and prints the contract's line: impl, metric, value, unit, the
    cpu_baseline it describes and an e2e with zero copies."""
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1", "--side", "64"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["config"]["L"] == 64 and "L=64" in d["config"]["note"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "L=64" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
