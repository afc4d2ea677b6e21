"""bench.py's clock sampler against a stand-in for nvidia-smi (a shell loop that prints the query's
CSV rows with a time stamp): the sampler is running before the timed region starts, rows stamped
before the region are left out, and the median SM clock, the maximum and the active throttle
reasons come from the rest."""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

STAMP = "$(date '+%Y/%m/%d %H:%M:%S.%3N')"


def _fake_smi(tmp_path, monkeypatch, clock_file, tail):
    """nvidia-smi stand-in: every 50 ms one row whose SM clock is read from clock_file."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\nwhile true; do "
                    f"echo \"{STAMP}, 0, $(cat {clock_file}), 2070, 900.0, {tail}\"; sleep 0.05; done\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")


def test_rows_before_the_timed_region_are_left_out(tmp_path, monkeypatch):
    clk = tmp_path / "clk"
    clk.write_text("810")                                      # idle GPU while the sampler starts
    _fake_smi(tmp_path, monkeypatch, clk, "0x4, Not Active, Not Active, Not Active, Active")
    c = bench.Clocks(0)
    c.wait_ready()
    assert os.path.getsize(c.f.name) > 0                       # sampling when the region starts
    time.sleep(0.3)
    clk.write_text("2055")
    time.sleep(0.06)
    c.mark()
    time.sleep(0.6)
    r = c.stop()
    assert r["samples"] >= 2
    assert r["sm_mhz"] == 2055.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_sampler_reports_a_thermal_slowdown(tmp_path, monkeypatch):
    clk = tmp_path / "clk"
    clk.write_text("1500")
    _fake_smi(tmp_path, monkeypatch, clk, "0x40, Not Active, Active, Not Active, Not Active")
    c = bench.Clocks(0)
    c.wait_ready()
    c.mark()
    time.sleep(0.3)
    r = c.stop()
    assert r["sm_mhz"] == 1500.0 and r["reasons"] == ["hw_thermal_slowdown"]


def test_unmarked_sampler_counts_every_row(tmp_path, monkeypatch):
    clk = tmp_path / "clk"
    clk.write_text("1980")
    _fake_smi(tmp_path, monkeypatch, clk, "0x0, Not Active, Not Active, Not Active, Not Active")
    c = bench.Clocks(0)
    c.wait_ready()
    time.sleep(0.2)
    r = c.stop()
    assert r["samples"] >= 2 and r["sm_mhz"] == 1980.0 and r["reasons"] == []


def test_wait_is_bounded_when_nothing_is_printed(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\nexec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = bench.Clocks(0)
    t0 = time.time()
    c.wait_ready(timeout_s=0.5)
    assert time.time() - t0 < 2.0
    r = c.stop()
    assert r["samples"] == 0 and r["sm_mhz"] is None
