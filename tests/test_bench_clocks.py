"""bench.py's clock record on a host without a GPU: a stand-in `nvidia-smi`
on PATH prints the CSV rows the real one prints under
`--query-gpu=... --format=csv,noheader,nounits -lms 100`, and the sampler
must turn them into the median SM clock, the maximum, and the active
throttle reasons; without any nvidia-smi it records nothing."""
import os
import stat
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FAKE = """#!/bin/sh
echo "0, 2070, 2070, 612.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
echo "0, 1980, 2070, 1391.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
echo "0, 2055, 2070, 1201.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
exec sleep 30
"""


def test_clock_record_from_the_sampler_rows(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE)
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    c = bench.ClockSampler(0)
    c.start()
    rec = c.stop()
    assert rec == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert c.proc.poll() is not None  # the sampler was ended


def test_no_sampler_no_record(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop() is None
