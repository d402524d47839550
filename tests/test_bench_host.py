"""Host-side logic of bench.py (no GPU): the reference arm's JSON line, the lookup of committed
ncu traffic stamps, and the roofline arithmetic."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    """--impl reference times the oracle on the host and prints one JSON line with the keys the
    driver reads (here on a 64^2 grid, one step)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "64",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["same_config"] is True


def test_traffic_stamp_is_used_only_while_the_kernel_sources_are_unchanged(tmp_path, monkeypatch):
    kernel = "k_fused2d_comp_nc2"
    stamp = os.path.join(ROOT, "profiles", f"traffic_{kernel}_rotation1024_f32.json")
    d = json.load(open(stamp))
    assert d["sources_sha256"] == bench.kernel_sources_sha256(kernel)
    assert bench.traffic_from_profiles(kernel, 1024, "f32") == d["bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda k: "0" * 64)
    assert bench.traffic_from_profiles(kernel, 1024, "f32") is None
    assert bench.traffic_from_profiles("no_such_kernel", 1024, "f32") is None


def test_fp64_and_alu_roofline_arithmetic():
    rates = {"f64_fma_per_s": 0.5e12, "f32_fma_per_s": 38e12, "how": "test"}
    r = bench.fp64_roofline(4e9, "2d", rates)
    assert r["frac"] == pytest.approx(4e9 * bench.FP64_OPS_PER_CELL_STEP["2d"] / 0.5e12, rel=1e-3)
    a = bench.alu_roofline(1 << 20, 20e-6, "k_fused2d_comp_nc2", 1024, "f32", 2070.0, 152, "compensated")
    peak = 152 * 128 * 2070e6 / 1e12
    assert a["peak"] == pytest.approx(peak, rel=1e-3)
    assert a["frac"] == pytest.approx(139 * (1 << 20) / 20e-6 / 1e12 / peak, rel=1e-3)
    assert bench.alu_roofline(1 << 20, 20e-6, "k", 1024, "f64", 2070.0, 152) is None
