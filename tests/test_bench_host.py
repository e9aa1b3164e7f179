"""Host logic of bench.py (CPU): the clock record that decides whether a timed
run is valid, the workload accounting, and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(sm, mx, reasons=("Not Active",) * 4):
    # index, clocks.sm, clocks.max.sm, power.draw, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    return ", ".join(["0", str(sm), str(mx), "900.0", "0x0"] + list(reasons))


def test_clocks_summary_median_and_reasons():
    c = bench.Clocks(0)
    c.lines = [_line(2032, 2032), _line(1980, 2032), _line(2032, 2032),
               _line(1800, 2032, ("Not Active", "Not Active", "Not Active", "Active")),
               "garbage line", ""]
    s = c.summary()
    assert s["samples"] == 4
    assert s["sm_mhz"] == 2006.0 and s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clocks_summary_flags_thermal_and_hw_slowdown():
    c = bench.Clocks(0)
    c.lines = [_line(1500, 2032, ("Active", "Not Active", "Active", "Not Active"))]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clocks_summary_without_samples():
    c = bench.Clocks(0)
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}


def test_workload_accounting():
    assert bench.dofs_per_element(3, 3) == 5 * 16 + 3 * 16 == 128
    assert bench.dofs_per_element(3, 2) == 5 * 16 + 3 * 9
    assert bench.vol_flops_per_element_pairs(3) == 117 * 48
    assert bench.vol_flops_per_element_minimal(3) == 4600
    assert bench.whole_job_value(2, 1000, 10, 1000.0) == 2 * 1000 * 10 / 1.0
    cfg = bench.workload_config(bench.STAB)
    assert cfg["workload"] == "orszag_tang_256x256_p3k3" and cfg["dofs_per_element"] == 128


def test_reference_arm_line():
    """The reference arm (the oracle on the host, bounded sample) prints one
    JSON line with the contract's keys; the warm-up is raised to 3."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["warmup"] == 3 and d["steps"] == 1
    assert d["value"] > 0 and d["unit"] == "DOF-updates/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_step_work_accounting():
    """Per-class algorithmic work of a Strang step: every class present,
    positive, the volume class equal to 6 launches of the minimal count, and
    the stabilisation statistics growing with the number of fields."""
    w = bench.step_work(3, 3)
    assert set(w) == {"face", "vol", "stab_hydro", "exchange", "mag_stage", "stab_eta", "stab_vel"}
    assert all(f > 0 and b > 0 for f, b in w.values())
    assert w["vol"][0] == 6 * bench.vol_flops_per_element_minimal(3)
    assert w["face"][0] == 6 * 2 * 4 * 70
    assert bench.stats_flops(3, 5) > bench.stats_flops(3, 3) > 0
    assert bench.step_work(4, 4)["vol"][0] > w["vol"][0]


def test_kernel_rooflines_bound_and_fraction():
    """A class timed exactly at its FP64 bound reads frac 1 and bound fp64;
    the step bound is the sum over classes of the larger time."""
    w = bench.step_work(3, 3)
    K, steps, p64, bw = 1000, 4, 1.0, 1000.0
    kt = {}
    for cls, (fl, by) in w.items():
        t = max(fl * K / (p64 * 1e12), by * K / (bw * 1e9)) * 1e3  # ms per step at the bound
        kt[cls] = (t * steps, 2 * steps)
    out, bound_ms = bench.kernel_rooflines(kt, K, steps, 3, 3, p64, bw)
    for cls, r in out.items():
        assert abs(r["frac"] - 1.0) < 1e-12
    assert out["vol"]["bound"] == "fp64"
    assert abs(bound_ms - sum(v[0] for v in kt.values()) / steps) < 1e-12


def test_workload_config_headline():
    cfg = bench.workload_config(bench.STAB, "blast")
    assert cfg["workload"] == "blast_1024x1024_p3k3" and cfg["gamma"] == 1.4 and cfg["mesh"] == [1024, 1024]
