"""The clock record of bench.py: nvidia-smi samples are kept only while the timed region is
open, and the throttle reasons are read from the query's columns.  A fake nvidia-smi on PATH
stands in for the GPU's (a shell loop that prints one query line every 50 ms)."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def fake_smi(tmp_path, line):
    p = tmp_path / "nvidia-smi"
    p.write_text(f"#!/bin/sh\nwhile true; do echo '{line}'; sleep 0.05; done\n")
    p.chmod(p.stat().st_mode | stat.S_IXUSR | stat.S_IXGRP | stat.S_IXOTH)
    return str(tmp_path)


@pytest.fixture
def bench_mod():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_samples_inside_the_window_only(tmp_path, monkeypatch, bench_mod):
    d = fake_smi(tmp_path, "0, 1980, 2070, 900.00, 0x4, Not Active, Not Active, Not Active, Active")
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ["PATH"])
    clk = bench_mod.ClockSampler(0)
    clk.start()
    assert clk.lines, "start() returns once the first sample has arrived"
    time.sleep(0.5)                       # before the window: not counted
    n_before = len(clk.lines)
    clk.begin()
    time.sleep(0.6)
    clk.end()
    time.sleep(0.3)                       # after the window: not counted
    rec = clk.stop()
    assert rec is not None
    assert 3 <= rec["samples"] <= 0.6 / 0.05 + 2
    assert rec["samples"] < len(clk.lines) - n_before + 1
    assert rec["sm_mhz"] == 1980.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert 0.55 <= rec["window_s"] <= 1.0


def test_throttle_reasons_are_reported(tmp_path, monkeypatch, bench_mod):
    d = fake_smi(tmp_path, "0, 1400, 2070, 1300.00, 0x48, Not Active, Active, Not Active, Not Active")
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ["PATH"])
    clk = bench_mod.ClockSampler(0)
    clk.start()
    clk.begin()
    time.sleep(0.3)
    clk.end()
    rec = clk.stop()
    assert rec["reasons"] == ["hw_thermal_slowdown"]
    assert rec["sm_mhz"] == 1400.0


def test_no_nvidia_smi(tmp_path, monkeypatch, bench_mod):
    monkeypatch.setenv("PATH", str(tmp_path))   # an empty directory: nvidia-smi is not found
    clk = bench_mod.ClockSampler(0)
    clk.start()
    clk.begin()
    clk.end()
    assert clk.stop() is None
