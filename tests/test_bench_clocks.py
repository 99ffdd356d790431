"""The clock record of bench.py's timed region, from a stand-in nvidia-smi on the CPU: the median
SM clock under load, the maximum clock, the sample count and the throttle reasons seen Active;
without nvidia-smi the record says so instead of failing the run."""
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

SAMPLES = [
    "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 1905, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2070, 2070, 1010.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "[N/A], [N/A]",  # a malformed line is skipped
]


def _fake_smi(tmp_path, lines):
    fake = tmp_path / "nvidia-smi"
    body = "".join(f"echo '{ln}'\n" for ln in lines)
    fake.write_text("#!/bin/sh\n" + body + "exec sleep 30\n")
    fake.chmod(0o755)
    return fake


def _run(monkeypatch, path_dirs, nlines=0):
    import bench
    monkeypatch.setenv("PATH", os.pathsep.join(path_dirs))
    c = bench.Clocks(0)
    c.start()
    if c.proc is not None:  # let the stand-in write its lines
        t0 = time.time()
        while time.time() - t0 < 10:
            with open(c.path) as f:
                if len(f.read().splitlines()) >= nlines:
                    break
            time.sleep(0.05)
    return c, c.stop()


def test_clock_record_from_samples(tmp_path, monkeypatch):
    _fake_smi(tmp_path, SAMPLES)
    c, r = _run(monkeypatch, [str(tmp_path), "/usr/bin", "/bin"], len(SAMPLES))
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(c.path)


def test_thermal_slowdown_is_reported(tmp_path, monkeypatch):
    _fake_smi(tmp_path, ["0, 1500, 2070, 1300.0, 0x40, Not Active, Active, Not Active, Not Active"])
    _, r = _run(monkeypatch, [str(tmp_path), "/usr/bin", "/bin"], 1)
    assert r["reasons"] == ["hw_thermal_slowdown"] and r["sm_mhz"] == 1500.0


def test_missing_nvidia_smi_is_recorded(tmp_path, monkeypatch):
    c, r = _run(monkeypatch, [str(tmp_path)])
    assert c.proc is None
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]
    assert not os.path.exists(c.path)
