"""Host pieces of the benchmark line, without a GPU: the algorithmic bytes of
the roofline's sweep, the reading of the clock samples taken during the
timed region (median SM clock, the largest maximum clock, every throttle
reason seen active), the peak's source, the defaults of a plain run, the
benchmark workload with its solver, and the combined device checks."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_algorithmic_bytes_of_one_viscous_sweep():
    # u_d read and written, rhs_d, the diagonal (or its inverse), mu_c, and per
    # other axis an edge viscosity and the other component
    cells = 128 * 128 * 256
    assert bench.alg_bytes_visc_sweep(3, cells, 4) == 36 * cells == 150994944
    assert bench.alg_bytes_visc_sweep(3, cells, 8) == 72 * cells
    assert bench.alg_bytes_visc_sweep(2, 64 * 32, 8) == 7 * 8 * 64 * 32


def clocks_from(tmp_path, lines):
    c = bench.Clocks(0)
    p = tmp_path / "clocks.csv"
    p.write_text("".join(line + "\n" for line in lines))
    c.path = str(p)
    return c.summary()


def test_clock_samples_are_summarised(tmp_path):
    ok = "Not Active"
    out = clocks_from(tmp_path, [
        "0, 2070, 2070, 900.1, 0x0, %s, %s, %s, %s" % (ok, ok, ok, ok),
        "0, 2060, 2070, 1390.5, 0x4, %s, %s, %s, Active" % (ok, ok, ok),
        "0, [N/A], 2070, 100.0, 0x0, %s, %s, %s, %s" % (ok, ok, ok, ok),   # skipped
        "0, 1900, 2070",                                                    # short: skipped
        "0, 1950, 2070, 1400.0, 0x8, Active, %s, %s, %s" % (ok, ok, ok),
    ])
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2060.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_no_clock_samples_is_said(tmp_path):
    out = clocks_from(tmp_path, [])
    assert out["sm_mhz"] is None and out["reasons"] == ["no samples"]


def test_the_peak_falls_back_when_no_measurement_is_present(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, src = bench.measured_peak()
    assert peak == 6800.0 and src.startswith("fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6795.8}')
    peak, src = bench.measured_peak()
    assert peak == pytest.approx(6795.8) and src.startswith("measured")


def test_defaults_are_one_gpu_and_a_short_run(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.impl == "ours" and a.config == "c3"
    assert a.warmup >= 3 and 1 <= a.steps <= 50
    assert a.solver == "tol"


def test_the_benchmark_workload_and_its_solver(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    inst = bench.load_workload("c3", None, a)
    p = inst["params"]
    # the 128x128x256 duct with 20,000 nodes, solved to relative residual
    # 1e-11 with the divergence target of 1e-10
    assert list(p["n"][:3]) == [128, 128, 256] and inst["X"].shape[0] == 20000
    assert p["vc_visc"] == 0 and p["vc_p"] == 0 and p["rtol"] == 1e-11
    assert p["div_tol"] == 1e-10 and p["precision"] == 1
    cfg = bench.describe(inst)
    assert cfg["cells"] == 128 * 128 * 256
    assert cfg["workload"].startswith("c3: 128x128x256 grid, 20000 nodes")
    assert "1e-11" in cfg["solver"]


def test_device_checks_of_several_simulations_are_combined():
    stats = [{"div_max_steps": 3e-11, "div_violations": 0, "nonconv_total": 1},
             {"div_max_steps": 9e-11, "div_violations": 2, "nonconv_total": 0}]
    assert bench.div_summary(stats) == {"div_max_all_steps": 9e-11, "div_violations": 2,
                                        "nonconverged_solves": 1}
