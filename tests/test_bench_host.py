"""Host logic of bench.py, on the CPU: the clock sampler keeps only the nvidia-smi lines
that arrive during the timed region.  A fake nvidia-smi on PATH stands in for the tool."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = """#!/bin/sh
# first 0.4 s: a low clock with hw_slowdown active; afterwards: full clock, no reason
start=$(date +%s%N)
while true; do
  now=$(date +%s%N)
  if [ $((now - start)) -lt 400000000 ]; then
    echo "0, 1000, 2070, 300.0, 0x8, Active, Not Active, Not Active, Not Active"
  else
    echo "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
  fi
  sleep 0.05
done
"""


@pytest.fixture
def fake_smi(tmp_path, monkeypatch):
    path = tmp_path / "nvidia-smi"
    path.write_text(FAKE)
    path.chmod(path.stat().st_mode | stat.S_IXUSR | stat.S_IXGRP | stat.S_IXOTH)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")
    return path


def _bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench

    return bench


def test_sampler_keeps_only_the_timed_region(fake_smi):
    b = _bench()
    s = b.ClockSampler(0)
    s.start()
    time.sleep(0.7)          # warm-up: the slow-clock lines arrive here
    s.mark_start()
    time.sleep(0.5)          # timed region
    s.mark_end()
    out = s.stop()
    assert out["samples"] >= 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == []


def test_sampler_reports_a_throttle_inside_the_region(fake_smi):
    b = _bench()
    s = b.ClockSampler(0)
    s.start()
    s.mark_start()
    time.sleep(0.3)          # the fake tool's slow, throttled phase
    s.mark_end()
    out = s.stop()
    assert out["samples"] >= 1 and "hw_slowdown" in out["reasons"]


def test_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    b = _bench()
    s = b.ClockSampler(0)
    s.start()
    s.mark_start()
    s.mark_end()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
