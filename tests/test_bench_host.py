"""Host-side logic of bench.py that needs no GPU: the clock / throttle-reason
sampler (against a fake nvidia-smi on PATH) and the panel's DRAM-traffic
figure, which is reported only for the kernel source it was measured on."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _fake_smi(tmp_path, lines):
    script = tmp_path / "nvidia-smi"
    body = "\n".join(f"echo '{l}'" for l in lines)
    script.write_text("#!/bin/sh\n" + body + "\nexec sleep 30\n")
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def _sample(monkeypatch, tmp_path, lines):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, lines) + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(0)
    c.start()
    time.sleep(0.5)
    return c.stop()


def test_clock_sampler_median_and_power_cap(monkeypatch, tmp_path):
    lines = ["0, 2070, 2070, 910.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1180.5, 0x0, Not Active, Not Active, Not Active, Not Active"]
    got = _sample(monkeypatch, tmp_path, lines)
    assert got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0 and got["samples"] == 3
    assert got["reasons"] == ["sw_power_cap"]


def test_clock_sampler_reports_thermal_slowdown(monkeypatch, tmp_path):
    lines = ["0, 1600, 2070, 1390.0, 0x20, Not Active, Not Active, Active, Not Active",
             "0, 1500, 2070, 1390.0, 0x48, Active, Active, Not Active, Not Active",
             "garbage line"]
    got = _sample(monkeypatch, tmp_path, lines)
    assert got["samples"] == 2 and got["sm_mhz"] == 1550.0
    assert got["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop()["reasons"] == ["unavailable"]


def test_panel_traffic_only_for_the_measured_source(monkeypatch):
    t = bench.panel_traffic_per_launch(4096)
    # the committed capture matches the committed kernel: 21st panel (2816 rows)
    # scaled to the average panel of N = 4096 (2080 rows)
    assert t is not None
    assert abs(t - bench.PANEL_TRAFFIC["bytes"] * 2080 / 2816) < 1e-6
    monkeypatch.setitem(bench.PANEL_TRAFFIC, "sha256", "0" * 64)
    assert bench.panel_traffic_per_launch(4096) is None
