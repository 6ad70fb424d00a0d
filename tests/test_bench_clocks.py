"""The benchmark's clock record keeps the nvidia-smi samples taken inside the
timed region (no GPU): throttle reasons and clocks outside the region do not
count, and unparsable timestamps fall back to every sample."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(ts, sm, reasons=("Not Active",) * 4):
    stamp = ts.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([stamp, "0", str(sm), "2070", "900.0", "0x0"] + list(reasons)) + "\n"


def test_samples_inside_the_timed_region_only():
    t0 = datetime.datetime(2026, 1, 2, 3, 4, 5, 0)
    lines = [_line(t0, 1200, ("Active", "Not Active", "Not Active", "Not Active")),   # warm-up, throttled
             _line(t0 + datetime.timedelta(milliseconds=100), 2070),
             _line(t0 + datetime.timedelta(milliseconds=120), 2070),
             _line(t0 + datetime.timedelta(milliseconds=140), 2055, ("Not Active",) * 3 + ("Active",)),
             _line(t0 + datetime.timedelta(milliseconds=400), 900)]                       # after the region
    on = (t0 + datetime.timedelta(milliseconds=90)).timestamp()
    off = (t0 + datetime.timedelta(milliseconds=150)).timestamp()
    out = bench.ClockSampler.summarise(lines, on, off)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    # no window: every sample
    everything = bench.ClockSampler.summarise(lines)
    assert everything["samples"] == 5 and everything["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_unparsable_timestamps_fall_back_to_every_sample():
    lines = ["N/A, 0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
             "N/A, 0, 2040, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
             "garbage\n"]
    out = bench.ClockSampler.summarise(lines, 0.0, 1.0)
    assert out["samples"] == 2 and out["sm_mhz"] == 2055.0 and out["reasons"] == []
