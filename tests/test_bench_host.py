"""Host logic of bench.py (no GPU): the roofline figures, the precision-form
Gram's executed-rate rule, and the clock-sample summary that decides whether
a run is kept."""
import pytest

import bench


def _prof(**ph):
    base = {k: {"ms": 0.0, "launches": 0, "calls": 0, "flops": 0.0, "bytes": 0.0}
            for k in ("transport", "gram_right", "eig", "gram_left", "small", "update", "energy")}
    for k, v in ph.items():
        base[k].update(v)
    return base


def test_roofline_takes_the_dominant_phase_and_divides_by_its_time():
    prof = _prof(gram_left={"ms": 2000.0, "launches": 40, "calls": 20, "flops": 1.6e12},
                 eig={"ms": 100.0, "launches": 10, "calls": 10})
    name, roof = bench.roofline_of(prof, 1.0, {"hbm_gbs": 7000.0})
    assert name == "gram_left" and roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    assert roof["achieved"] == pytest.approx(0.8)
    assert roof["frac"] == pytest.approx(0.8) and roof["avg_phase_ms"] == pytest.approx(100.0)
    assert roof["traffic"] == pytest.approx(bench.GRAM_LEFT_CAP_TRAFFIC)


def test_roofline_of_a_bandwidth_phase_uses_the_measured_copy_rate():
    prof = _prof(transport={"ms": 10.0, "launches": 5, "calls": 5, "bytes": 3.5e10})
    name, roof = bench.roofline_of(prof, 1.0, {"hbm_gbs": 7000.0})
    assert name == "transport" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(3500.0) and roof["frac"] == pytest.approx(0.5)
    assert roof["traffic"] is None


def test_precision_form_gram_counts_28_digit_products_per_term():
    gl = {"ms": 1000.0, "flops": 1e13}
    r = bench.tc_gram_roofline(gl, {"bf16_tflops_sustained": 1400.0, "bf16_tflops": 1900.0})
    assert r["achieved"] == pytest.approx(280.0) and r["frac"] == pytest.approx(0.2)
    assert r["fp64_equivalent_tflops"] == pytest.approx(10.0)
    assert bench.tc_gram_roofline({"ms": 0.0, "flops": 1.0}, {}) is None


def test_clock_summary_reports_median_and_active_reasons():
    rows = ["0, 2032, 2070, 1100.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2070, 2070, 1190.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2070, 1250.0, 0x4, Not Active, Not Active, Not Active, Active",
            "garbage line"]
    c = bench.parse_clock_rows(rows)
    assert c["sm_mhz"] == 2032 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"] and c["power_w_median"] == 1190.0
    hot = bench.parse_clock_rows(["0, 1500, 2070, 900, 0x40, Not Active, Active, Not Active, Not Active"])
    assert hot["reasons"] == ["hw_thermal_slowdown"]
    assert bench.parse_clock_rows([]) is None


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle timed on the host) prints one
    JSON line with the arm's fields, on a CPU-only machine."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-budget", "5"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
