"""bench.py's host-side helpers: the nvidia-smi clock sampler of the timed
region, run here against a stand-in nvidia-smi that prints fixed samples."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FAKE = """#!/bin/sh
echo "1965, 2070, 1105.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
echo "2032, 2070, 980.7, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
echo "1998, 2070, 1010.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
echo "[N/A], 2070, 1010.0, 0x0, Not Active, Not Active, Not Active, Not Active"
sleep 30
"""


def _fake_smi(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE)
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")


def _sample(clk):
    with clk:
        deadline = time.time() + 10
        while time.time() < deadline and os.path.getsize(clk.path) < 200:
            time.sleep(0.05)
    return clk.summary()


def test_clock_summary_median_max_and_reasons(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch)
    clk = bench.Clocks(0)
    s = _sample(clk)
    assert s == {"sm_mhz": 1998.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not os.path.exists(clk.path)          # the temporary file is removed


def test_clock_samples_kept_when_a_path_is_given(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch)
    out = tmp_path / "out" / "clocks.csv"
    s = _sample(bench.Clocks(0, str(out)))
    assert s["samples"] == 3
    assert len(out.read_text().splitlines()) == 4


def test_no_nvidia_smi_gives_no_clocks(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    clk = bench.Clocks(0)
    with clk:
        pass
    assert clk.summary() is None
    assert not os.path.exists(clk.path)
