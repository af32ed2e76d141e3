"""Host-side logic of bench.py that needs no GPU: the clock / throttle-reason
sampler (against a fake nvidia-smi on PATH), the tensor-core roofline's
arithmetic on a synthetic per-kernel profile, and the DRAM-traffic figure,
which is reported only for the kernel source it was measured on."""
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


def test_trailing_update_flops_is_two_thirds_n_cubed():
    # sum over block steps of 2 m^2 nb, m = n - j - nb: ~ 2 n^3 / 3 for n >> nb
    assert bench.trailing_update_flops(128, 64) == 2.0 * 64 ** 2 * 64
    f = bench.trailing_update_flops(8192)
    assert abs(f / (2 * 8192 ** 3 / 3) - 1) < 0.02


def test_group_update_flops():
    # n = 3 groups of 2 block steps (nb = 64): groups 0 and 1 have far columns
    n = 6 * 64
    f = bench.group_update_flops(n, 2)
    want = 2.0 * (n - 128) * (n - 192) * 128 + 2.0 * (n - 256) * (n - 320) * 128
    assert f == want
    # the group launches carry most of the update; never more than all of it
    for g in (1, 4, 8, 16):
        assert bench.group_update_flops(8192, g) < bench.trailing_update_flops(8192)
    assert bench.group_update_flops(8192, 8) > 0.8 * bench.trailing_update_flops(8192)


def test_tensor_roofline_is_per_step_not_per_run():
    """The profile sums every launch of every profiled step; the roofline divides
    one factorization's flops by one step's kernel time, so the result does not
    depend on how many steps were profiled."""
    n, peaks = 8192, {"bf16_tflops": 2000.0, "source": "measured"}
    flops = bench.group_update_flops(n, 4)
    per_step_ms, per_step_calls = 2.0, 31
    for steps in (1, 5, 20):
        prof = {"gemm_tc_group": (per_step_ms * steps, per_step_calls * steps), "panel": (10.0 * steps, 128 * steps)}
        r = bench.tensor_roofline(prof, steps, n, peaks, 4)
        assert abs(r["achieved"] - flops / 2e-3 / 1e12) < 1e-9 * r["achieved"]
        assert abs(r["frac"] - r["achieved"] / 2000.0) < 1e-15
        assert r["launches_per_step"] == per_step_calls
        assert abs(r["avg_launch_ms"] - per_step_ms / per_step_calls) < 1e-15
        # per launch: flops of an average launch over its average duration
        assert abs(r["flops_per_launch"] / (r["avg_launch_ms"] * 1e-3) / 1e12 - r["achieved"]) < 1e-6
    assert bench.tensor_roofline({"panel": (1.0, 1)}, 1, n, peaks, 4) is None


def test_traffic_only_for_the_measured_source(tmp_path, monkeypatch):
    import hashlib
    import json
    src = tmp_path / "k.cu"
    src.write_text("kernel source")
    rec = {"k_gemm_tc": {"source": str(src), "sha256": hashlib.sha256(b"kernel source").hexdigest(),
                         "bytes_per_launch": 1234.5}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.traffic_per_launch("k_gemm_tc") == 1234.5
    assert bench.traffic_per_launch("k_panel") is None
    src.write_text("kernel source, changed")
    assert bench.traffic_per_launch("k_gemm_tc") is None
