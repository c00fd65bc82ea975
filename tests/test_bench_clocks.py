"""The bench's clock sampler (host logic): it parses nvidia-smi's CSV
samples into the median SM clock, the largest maximum and the throttle
reasons seen, waits for the first sample before the timed region starts,
and degrades to "unavailable" without nvidia-smi.  A stand-in nvidia-smi
script on PATH plays the tool; no GPU is involved."""
from __future__ import annotations

import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _fake_smi(tmp_path, lines, period=0.05):
    body = "".join(f'echo "{ln}"\n' for ln in lines)
    script = tmp_path / "nvidia-smi"
    script.write_text(f"#!/bin/sh\nsleep 0.2\nwhile true; do\n{body}sleep {period}\ndone\n")
    script.chmod(0o755)
    return script


def test_sampler_median_max_and_reasons(tmp_path, monkeypatch):
    _fake_smi(tmp_path, ["0, 2070, 2070, 900.5, 0x4, Not Active, Not Active, Not Active, Active",
                         "0, 1950, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                         "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active"])
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    s = bench.ClockSampler(0)
    t0 = time.perf_counter()
    s.start()
    waited = time.perf_counter() - t0
    # the sampler returns once the first sample is there (the stand-in
    # starts after 0.2 s), well before its 3 s limit
    assert 0.15 < waited < 2.5
    time.sleep(0.3)
    c = s.stop()
    assert c["samples"] >= 3
    assert c["sm_mhz"] == 2070.0
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_sampler_flags_thermal_slowdown(tmp_path, monkeypatch):
    _fake_smi(tmp_path, ["0, 1500, 2070, 1400.0, 0x40, Not Active, Active, Not Active, Not Active"])
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.15)
    c = s.stop()
    assert c["sm_mhz"] == 1500.0
    assert c["reasons"] == ["hw_thermal_slowdown"]


def test_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # an empty directory: no tool
    s = bench.ClockSampler(0)
    s.start()
    c = s.stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]
