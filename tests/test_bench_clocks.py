"""The bench's clock record (host logic, no GPU): bench.ClockSampler reads
nvidia-smi's stamped samples, keeps those stamped inside the timed region
marked by begin()/end(), and reports throttle reasons.  A fake nvidia-smi on
PATH prints samples every 20 ms in nvidia-smi's CSV form."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FAKE = r'''#!/usr/bin/env python3
import sys, time
from datetime import datetime
mhz = "{mhz}"
reason = "{reason}"
i = 0
while True:
    ts = datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    cap = reason if i % 3 == 0 else "Not Active"
    print(f"{{ts}}, 0, {{mhz}}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, {{cap}}", flush=True)
    i += 1
    time.sleep(0.02)
'''


def _install(tmp_path, monkeypatch, mhz="2070", reason="Not Active"):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE.format(mhz=mhz, reason=reason))
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")


def test_samples_inside_the_region(tmp_path, monkeypatch):
    _install(tmp_path, monkeypatch)
    c = bench.ClockSampler(0)
    time.sleep(0.15)                              # samples before the region
    c.begin()
    time.sleep(0.3)
    c.end()
    time.sleep(0.15)                              # and after it
    r = c.stop()
    assert r["in_region"] and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert 5 <= r["samples"] <= 20                # about 15 samples of 20 ms in 300 ms
    assert r["reasons"] == [] and 290 <= r["region_ms"] <= 400


def test_reasons_and_short_region(tmp_path, monkeypatch):
    _install(tmp_path, monkeypatch, mhz="1500", reason="Active")
    c = bench.ClockSampler(0)
    c.begin()
    c.end()                                       # shorter than one sampling interval
    time.sleep(0.2)
    r = c.stop()
    assert r["sm_mhz"] == 1500.0 and "sw_power_cap" in r["reasons"]
    assert r["samples"] >= 1                      # falls back to every sample of the run


def test_no_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))     # nothing to run
    c = bench.ClockSampler(0)
    c.begin()
    c.end()
    assert c.stop() is None


@pytest.mark.parametrize("text", ["2026/12/03 21:29:42.123", "garbage"])
def test_stamp_parsing(text):
    v = bench.ClockSampler._stamp(text)
    assert (v is None) == (text == "garbage")
