"""The benchmark's clock record: median and maximum SM clock and the throttle reasons
seen active during the timed region, parsed from nvidia-smi's CSV samples (a run
that saw a hardware or thermal slowdown is to be rejected, so the reasons must be
reported exactly)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clean_samples():
    out = "\n".join(f"0, {mhz}, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
                    for mhz in (2070, 2070, 1995, 2070, 2055))
    r = bench.ClockSampler.parse(out)
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}


def test_reasons_and_malformed_lines():
    out = "\n".join([
        "0, 1800, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1500, 2070, 1400.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Active, Not Active",
        "",
    ])
    r = bench.ClockSampler.parse(out)
    assert r["samples"] == 2 and r["sm_mhz"] == 1650.0 and r["sm_max_mhz"] == 2070.0
    # the sample whose clock reads N/A adds no clock, but its reasons count
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_no_samples():
    assert bench.ClockSampler.parse("") == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
