"""The benchmark's JSON contract and roofline arithmetic, on CPU: the
reference arm (the oracle on the host cores) prints one line with the
contract's keys; the roofline helper divides the documented algorithmic
bytes and flops per cell-update by the kernel time and the peak."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_one_contract_line():
    # a 4^3-patch box keeps the CPU run small; the line's keys do not depend on it
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--patches", "4"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["data"] == "synthetic"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_algorithmic_bytes_and_flops_per_cell_update():
    import bench
    # read and write 8 stored fields, plus the g = 3 guard shell of a 32^3
    # patch from one neighbour slice: ((38^3 - 32^3) / 32^3) * 8 values,
    # 171.2 B (FP64) and 85.6 B (FP32) per cell-update; the stencil's own
    # radius-2 shell beside it
    shell = (38 ** 3 - 32 ** 3) / 32 ** 3
    assert bench.alg_bytes_per_cell(32, 8) == pytest.approx(8 * (16 + shell * 8))
    assert bench.alg_bytes_per_cell(32, 8) == pytest.approx(171.2, abs=0.05)
    assert bench.alg_bytes_per_cell(32, 4) == pytest.approx(85.6, abs=0.05)
    assert bench.alg_bytes_per_cell(16, 8) == pytest.approx(230.4, abs=0.05)
    assert bench.alg_bytes_per_cell(24, 4, sbar=2) == pytest.approx(125.0, abs=0.05)
    shell2 = (36 ** 3 - 32 ** 3) / 32 ** 3
    assert bench.alg_bytes_radius2(32, 4) == pytest.approx(4 * (16 + shell2 * 8))
    assert bench.ALG_FLOPS_PER_CELL == 1424
    assert bench.ALG_FLOPS_PER_CELL_HLLD == 1424 + 3 * (170 - 37)


def test_roofline_fractions():
    import bench
    ncells, kernel_ms, hbm_peak = 16777216, 64.0, 6788.6
    r = bench.rooflines(ncells, 8, kernel_ms, hbm_peak, "measured")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    flops = bench.ALG_FLOPS_PER_CELL * ncells
    assert r["achieved"] == pytest.approx(flops / (kernel_ms * 1e-3) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["hbm"]["achieved"] == pytest.approx(bench.alg_bytes_per_cell(32, 8) * ncells / (kernel_ms * 1e-3) / 1e9)
    assert r["hbm"]["frac"] == pytest.approx(r["hbm"]["achieved"] / hbm_peak)
    r32 = bench.rooflines(ncells, 4, 4.5, hbm_peak, "measured")
    assert r32["bound"] == "hbm" and r32["alu"]["bound"] == "alu"
    assert r32["frac"] == pytest.approx(bench.alg_bytes_per_cell(32, 4) * ncells / 4.5e-3 / 1e9 / hbm_peak)
