"""Host-side helpers of bench.py: the clock-sample summary that decides
whether a timed run is kept (throttle reasons under load), the roofline
entry, and the Darcy permeability's normalisation."""
import numpy as np

import bench


def _line(sm, power, hw="Not Active", hwt="Not Active", swt="Not Active", swp="Not Active"):
    return f"0, {sm}, 2070, {power}, 0x0, {hw}, {hwt}, {swt}, {swp}"


def test_clock_summary_uses_samples_under_load():
    out = "\n".join([_line(1980, 120.0), _line(2070, 900.0), _line(2070, 950.0), _line(2055, 910.0),
                     "garbage line", _line(600, 80.0, hw="Active")])
    c = bench.Clocks.summarise(out)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["samples"] == 5 and c["samples_under_load"] == 3
    assert c["reasons"] == []  # the idle sample's hw_slowdown does not count
    assert c["power_w_max"] == 950.0


def test_clock_summary_reports_throttle_reasons():
    out = "\n".join([_line(1800, 1300.0, swp="Active"), _line(1700, 1350.0, hwt="Active"),
                     _line(1750, 1320.0, swt="Active")])
    c = bench.Clocks.summarise(out)
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert c["sm_mhz"] == 1750.0


def test_clock_summary_without_samples():
    assert bench.Clocks.summarise("") is None


def test_roofline_entry_fp32_and_fp64():
    r = bench.roofline_entry(6.0e9, 1.0e9, 1.0, 4, 6000.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 6000.0) < 1e-9 and abs(r["frac"] - 1.0) < 1e-12
    r64 = bench.roofline_entry(6.0e9, 0.63e9, 1.0, 8, 6000.0)
    assert r64["bound"] == "alu" and r64["unit"] == "TFLOP/s"
    assert abs(r64["achieved"] - 0.63) < 1e-12
    # without a measured FP64 rate the figure from unit counts stands in, and says so
    assert bench.FP64_PEAK["tflops"] is None
    assert abs(r64["frac"] - 0.63 / bench.FP64_PEAK_DERIVED_TFLOPS) < 1e-12
    assert r64["peak_source"].startswith("derived")
    bench.FP64_PEAK.update(tflops=1.25, source="measured: test")
    try:
        r64 = bench.roofline_entry(6.0e9, 0.63e9, 1.0, 8, 6000.0)
        assert abs(r64["frac"] - 0.63 / 1.25) < 1e-12 and r64["peak_source"] == "measured: test"
    finally:
        bench.FP64_PEAK.update(tflops=None, source=None)


def test_darcy_permeability_normalisation():
    """Uniform u_x = U on half of the nodes: q_D = U / 2, k = nu U / (2 g)."""
    class Geo:
        N = 8

    u = np.zeros((3, 8))
    u[0, :4] = 2e-4
    k = bench.darcy_permeability(Geo(), u, 0.1, 1e-6)
    assert abs(k - 0.1 * 1e-4 / 1e-6) < 1e-9


def test_oracle_baseline_is_timed_on_all_cores_and_on_one():
    """run_oracle (the bench's cpu_baseline): the FP64 oracle on a cube of the
    workload's recipe, every host core and then one thread, each run's step
    count set from a two-step timing; the entry carries the contract's keys."""
    import os

    out = bench.run_oracle(32, target_s=0.05, single_target_s=0.05)
    assert out["kind"] == "oracle" and out["unit"] == "MLUPS"
    assert out["value"] > 0 and out["cores"] == (os.cpu_count() or 1)
    assert out["single_thread"]["cores"] == 1 and out["single_thread"]["value"] > 0
    assert out["single_thread"]["steps"] >= 2
    assert "32^3 sub-case" in out["sample"] and "OpenMP threads" in out["sample"]
