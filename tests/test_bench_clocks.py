"""bench.py's clock sampler against a stand-in for nvidia-smi (a shell loop that prints the query's
CSV rows): the sampler is running before the timed region starts, the median SM clock, the maximum
and the active throttle reasons come from the rows it printed."""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _fake_smi(tmp_path, rows):
    body = "".join(f"echo '{r}'; sleep 0.05; " for r in rows)
    fake = tmp_path / "nvidia-smi"
    fake.write_text(f"#!/bin/sh\nwhile true; do {body}done\n")
    fake.chmod(0o755)
    return fake


def test_sampler_is_live_before_the_timed_region(tmp_path, monkeypatch):
    _fake_smi(tmp_path, ["0, 1965, 2070, 900.5, 0x4, Not Active, Not Active, Not Active, Active",
                         "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                         "0, 1980, 2070, 910.0, 0x4, Not Active, Not Active, Not Active, Active"])
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = bench.Clocks(0)
    c.wait_ready()
    assert os.path.getsize(c.f.name) > 0       # a sample exists when timing would start
    time.sleep(0.4)
    r = c.stop()
    assert r["samples"] >= 3
    assert r["sm_mhz"] in (1965.0, 1980.0, 2070.0) and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_sampler_reports_a_thermal_slowdown(tmp_path, monkeypatch):
    _fake_smi(tmp_path, ["0, 1500, 2070, 1390.0, 0x40, Not Active, Active, Not Active, Not Active"])
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = bench.Clocks(0)
    c.wait_ready()
    time.sleep(0.2)
    r = c.stop()
    assert r["sm_mhz"] == 1500.0 and r["reasons"] == ["hw_thermal_slowdown"]


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
