"""Host-side logic of bench.py that needs no GPU: the clock record and the
FFT flop model's plan lengths.

The benchmark reports the median SM clock and the throttle reasons that
nvidia-smi saw during the timed region; samples stamped outside that window
(start-up, warm-up, the copy-out afterwards) must not count.  Its FFT flop
count follows the lengths the library's compile-time plans run, so its copy
of those lengths must match the library's plan table.
"""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(ts, sm, reasons=("Not Active",) * 4):
    return ", ".join([ts.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3], "0", str(sm), "2070", "900.0", "0x0", *reasons])


def test_clock_record_keeps_only_the_timed_window():
    t = datetime.datetime(2026, 1, 2, 3, 4, 5)
    ms = datetime.timedelta(milliseconds=1)
    lines = [_line(t, 345), _line(t + 100 * ms, 2070), _line(t + 120 * ms, 2055), _line(t + 140 * ms, 2070),
             _line(t + 400 * ms, 600, ("Not Active", "Not Active", "Not Active", "Active"))]
    r = bench.parse_clock_lines(lines, t + 90 * ms, t + 150 * ms)
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == []
    every = bench.parse_clock_lines(lines)
    assert every["samples"] == 5 and every["reasons"] == ["sw_power_cap"]


def test_clock_record_flags_throttle_reasons_in_the_window():
    t = datetime.datetime(2026, 1, 2, 3, 4, 5)
    ms = datetime.timedelta(milliseconds=1)
    lines = [_line(t + 10 * ms, 1800, ("Active", "Not Active", "Active", "Not Active")),
             "garbage", "", _line(t + 30 * ms, 1900)]
    r = bench.parse_clock_lines(lines, t, t + 50 * ms)
    assert r["samples"] == 2 and r["sm_mhz"] == 1850.0
    assert r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_tool():
    s = bench.ClockSampler(0)
    assert s.stop()["samples"] == 0


def test_flop_model_uses_the_library_plan_lengths():
    """bench.FF_LENGTHS (the FFT flop model) lists exactly the lengths of the
    compile-time plans in the library's ST_FF_PLANS table."""
    import re
    src = open(os.path.join(ROOT, "paper_1908_06096_gb300", "csrc", "st_internal.cuh")).read()
    table = src[src.index("#define ST_FF_PLANS(X)"):]
    table = table[:table.index("constexpr int FF_NPLANS")]
    lengths = set()
    for m in re.finditer(r"X\((\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+)\)", table):
        a, b, c, d = (int(m.group(i)) for i in range(3, 7))
        lengths.add(a * b * c * d)
    n = int(re.search(r"constexpr int FF_NPLANS = (\d+);", src).group(1))
    assert len(re.findall(r"X\(\d+,", table)) == n
    assert sorted(lengths) == sorted(bench.FF_LENGTHS)
