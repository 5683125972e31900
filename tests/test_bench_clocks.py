"""bench.py's clock record: nvidia-smi samples are parsed, those inside the
timed region kept (or all of them if none is), the SM clock taken as the
median of the loaded samples and every throttle reason seen reported."""
import datetime

import bench


def _line(t: float, sm: int, mx: int = 2032, reasons=("Not Active",) * 4) -> str:
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([ts, str(sm), str(mx), "812.5", "0x0000000000000000", *reasons])


def _clocks(lines, t0, t1):
    c = bench.Clocks(0)
    c.t0, c.t1, c.lines = t0, t1, lines
    return c.summary()


def test_samples_inside_the_timed_region_only():
    t0 = 1_800_000_000.0
    lines = [_line(t0 - 1.0, 800), _line(t0 + 0.10, 2032), _line(t0 + 0.15, 2025), _line(t0 + 0.20, 2032),
             _line(t0 + 2.0, 900)]
    s = _clocks(lines, t0, t0 + 0.3)
    assert s["samples_in_timed_region"] == 3 and s["samples"] == 3
    assert s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2032.0 and s["reasons"] == []


def test_reasons_and_fallback_to_every_sample():
    t0 = 1_800_000_000.0
    hot = ("Not Active", "Active", "Not Active", "Active")  # hw thermal slowdown and the power cap
    lines = [_line(t0 - 1.0, 1500, reasons=hot), _line(t0 + 5.0, 2032)]
    s = _clocks(lines, t0, t0 + 0.1)  # no sample inside: every sample is used
    assert s["samples_in_timed_region"] == 0 and s["samples"] == 2
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["sm_mhz"] == 1766.0  # the median of the loaded samples (both above half the max)


def test_unreadable_output():
    assert _clocks(["no devices were found", ""], 0.0, 1.0) is None
