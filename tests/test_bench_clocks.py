"""bench.py's clock record: nvidia-smi samples are stamped when they arrive and
only those inside the timed region are summarised.  Runs on CPU against a fake
nvidia-smi that prints one idle line, then loaded lines every 50 ms."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = """#!/bin/bash
echo "0, 100, 2070, 50.0, 0x0, Not Active, Not Active, Not Active, Not Active"
while true; do
  sleep 0.05
  echo "0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active"
done
"""


def test_clock_sampler_keeps_only_the_timed_region(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text(FAKE)
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.start()
    assert c.lines, "start() returns once the first sample has arrived"
    t0 = time.perf_counter()            # the idle first line is stamped before the region
    time.sleep(0.4)
    t1 = time.perf_counter()
    r = c.stop(t0, t1)
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert r["samples"] >= 3 and r["interval_ms"] == bench.ClockSampler.INTERVAL_MS


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.start()
    r = c.stop(0.0, 1.0)
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]
