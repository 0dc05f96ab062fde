"""Host-side logic of bench.py on CPU: the clock sampler's reading of the
nvidia-smi CSV stream (a fake nvidia-smi on PATH prints fixed samples; no
GPU setting is read or changed), the traffic figure's validity guard, and
the roofline peak's source."""
import os
import time

import bench


def _fake_smi(tmp_path, lines):
    p = tmp_path / "nvidia-smi"
    body = "".join(f"echo '{ln}'\n" for ln in lines)
    p.write_text("#!/bin/sh\n" + body + "exec sleep 30\n")
    p.chmod(0o755)
    return str(tmp_path)


def _sample(cs, n):
    cs.start()
    deadline = time.time() + 10
    while len(cs.samples) < n and time.time() < deadline:
        time.sleep(0.02)
    return cs.stop()


def test_clock_sampler_median_max_and_reasons(tmp_path, monkeypatch):
    lines = [
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1300.2, 0x8, Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, lines) + os.pathsep + os.environ["PATH"])
    out = _sample(bench.ClockSampler(0), len(lines))
    assert out["samples"] == 4
    assert out["sm_mhz"] == 2070.0  # median of the readable SM clocks 2070, 1980, 2070
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_sampler_quiet_run_has_no_reasons(tmp_path, monkeypatch):
    lines = ["0, 1965, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active"] * 3
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, lines) + os.pathsep + os.environ["PATH"])
    out = _sample(bench.ClockSampler(0), 3)
    assert out["reasons"] == [] and out["sm_mhz"] == 1965.0


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # an empty directory
    cs = bench.ClockSampler(0)
    cs.start()
    out = cs.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_figure_only_for_the_captured_source(monkeypatch):
    """The committed DRAM figure is reported while the stream-collide source
    has the hash it was captured on, and null otherwise."""
    import json
    with open(os.path.join(bench.ROOT, "profiles", "step_f32_vec_traffic.json")) as fh:
        cap = json.load(fh)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: cap["kernel_source_sha256_16"])
    assert bench.profiled_traffic() == cap["dram_bytes_per_full_launch"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic() is None


def test_peak_source():
    """The measured copy bandwidth when the peaks file is there, else the
    stated fallback."""
    peak, kind = bench.measured_peaks()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and 1000.0 < peak < 10000.0
    else:
        assert kind == "fallback" and peak == bench.FALLBACK_HBM_GBS
