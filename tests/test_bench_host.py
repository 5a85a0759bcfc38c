"""Host-side logic of bench.py and the trajectory tool, on the CPU: the clock record that
decides whether a measurement is kept, the code-only hash that ties the recorded DRAM traffic to
a kernel source, and the drift / fluctuation statistics of a trajectory."""
import numpy as np
import pytest

import bench


def _line(sm, smax, active, hw="Not Active", hw_th="Not Active", sw_th="Not Active", pcap="Not Active"):
    return f"0, {sm}, {smax}, 900.00, {active}, {hw}, {hw_th}, {sw_th}, {pcap}"


def test_clock_summary_uses_timed_samples_only():
    lines = [(0.5, _line(1000, 2070, "0x4", hw="Active")),          # before the mark: ignored
             (1.0, _line(2070, 2070, "0x0")),
             (1.1, _line(2055, 2070, "0x0", pcap="Active")),
             (1.2, _line(2070, 2070, "0x0")),
             (1.3, "garbage line"),
             (1.4, _line("[N/A]", 2070, "0x0"))]
    r = bench.ClockSampler.summarise(lines, t_mark=1.0)
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]           # "Not Active" is not a reason


def test_clock_summary_reports_throttle_reasons():
    lines = [(2.0, _line(1500, 2070, "0x8", hw_th="Active", sw_th="Active"))]
    r = bench.ClockSampler.summarise(lines, t_mark=0.0)
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler.summarise([], 0.0) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                                                      "samples": 0}


def test_kernel_hash_ignores_comments_only():
    code = 'int f(int x) {\n  return x + 1;  // one\n}\n/* block\n comment */\nconst char* s = "a//b";\n'
    assert bench.strip_comments(code) == 'int f(int x) {\n  return x + 1;\n}\nconst char* s = "a//b";'
    assert bench.strip_comments(code.replace("// one", "// two\n\n")) == bench.strip_comments(code)
    assert bench.strip_comments(code.replace("x + 1", "x + 2")) != bench.strip_comments(code)


def test_kernel_hash_of_the_tree_is_stable():
    assert bench.kernel_sha1() == bench.kernel_sha1()
    assert len(bench.kernel_sha1()) == 40


def test_trajectory_drift_and_fluctuation():
    try:
        from paper_2606_03140_gb300 import md          # loads the library through the binding
    except Exception as e:                             # library not built on this machine
        pytest.skip(f"binding not loadable: {e}")
    n_atoms, dt_fs, steps = 100, 0.25, 4000
    t_ps = np.arange(steps) * dt_fs / 1000.0
    rng = np.random.default_rng(3)
    noise = 1e-3 * rng.standard_normal(steps)
    E = np.zeros((steps, 3))
    E[:, 2] = -50.0 + 2e-2 * t_ps + noise           # 2e-2 Ha/ps over 100 atoms
    st = md._energy_stats(E, n_atoms, dt_fs, skip=400)
    assert st["drift_ha_per_atom_ps"] == pytest.approx(2e-4, rel=0.05)
    assert st["fluct_rms_ha_per_atom"] == pytest.approx(1e-5, rel=0.05)
    assert st["fit_window_ps"][0] == pytest.approx(0.1)
