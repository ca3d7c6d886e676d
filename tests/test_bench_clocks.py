"""bench.py's clock record: the samples kept for a timed region shorter than
the sampling interval (the last one before it and the first one after), the
throttle reasons collected from them, and no record without samples."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _row(t, mhz, reasons=()):
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    return (t, float(mhz), 2032.0) + tuple("Active" if n in reasons else "Not Active" for n in names)


def test_short_region_keeps_the_bracketing_samples():
    base = datetime.datetime(2026, 1, 1, 12, 0, 0)
    s = lambda ms: base + datetime.timedelta(milliseconds=ms)  # noqa: E731
    rows = [_row(s(0), 1200), _row(s(500), 2032), _row(s(1000), 2032), _row(s(1500), 2032, ("sw_power_cap",)),
            _row(s(3000), 900, ("hw_slowdown",))]
    # a 35 ms region between samples at 1.0 s and 1.5 s
    c = bench.clock_summary(rows, s(1200), s(1235))
    assert c["samples"] == 2 and c["sm_mhz"] == 2032.0 and c["sm_max_mhz"] == 2032.0
    assert c["reasons"] == ["sw_power_cap"] and c["window_s"] == 0.5
    # samples inside the padded region are all kept, far ones are not
    c = bench.clock_summary(rows, s(450), s(1050))
    assert c["samples"] == 4 and "hw_slowdown" not in c["reasons"]
    assert bench.clock_summary([], s(0), s(1)) is None
