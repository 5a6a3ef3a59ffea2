"""The bench's host-side records (no GPU): the clock record (median SM clock
under load, the maximum, every throttle reason seen active in the samples) and
the host cores the CPU baseline may use."""
import tempfile
import types

import bench


def record(lines):
    c = bench.Clocks(0)
    c.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    c.f.write("\n".join(lines) + "\n")
    c.f.flush()
    c.proc = types.SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: 0, kill=lambda: None)
    return c.stop()


def test_median_max_and_active_reasons():
    got = record([
        "0, 2070, 2070, 610.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 700.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ])
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_slowdowns_are_reported_and_unreadable_rows_skipped():
    got = record([
        "0, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
        "0, 1200, 2070, 900.0, 0x08, Active, Not Active, Not Active, Not Active",
        "0, 1300, 2070, 900.0, 0x48, Active, Active, Not Active, Not Active",
        "",
    ])
    assert got["samples"] == 2 and got["sm_mhz"] == 1250.0
    assert got["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_no_samples_gives_no_record():
    assert record([]) is None
    assert bench.Clocks(0).stop() is None  # never started


def test_host_cores_lists_the_affinity_as_ranges(monkeypatch):
    monkeypatch.setattr(bench.os, "sched_getaffinity", lambda pid: {0, 1, 2, 5, 7, 8}, raising=False)
    monkeypatch.setattr(bench.os, "cpu_count", lambda: 16)
    assert bench.host_cores() == (16, 6, "0-2,5,7-8")
    monkeypatch.setattr(bench.os, "sched_getaffinity", lambda pid: {3}, raising=False)
    assert bench.host_cores() == (16, 1, "3")
