"""The benchmark's host-side pieces on the CPU: the clock record taken during
the timed region (median SM clock under load, maximum clock, which
throttle reasons were active) from nvidia-smi's CSV lines."""
import bench


def sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s.stop()


def row(sm, mx=2070, reasons=("Not Active",) * 4):
    return ", ".join(["0", str(sm), str(mx), "900.5", "0x0000000000000000", *reasons])


def test_clock_record():
    lines = [row(1965), row(1980), row(2010), "garbage", "", row("N/A"),
             row(1995, reasons=("Not Active", "Not Active", "Not Active", "Active"))]
    rec = sampler(lines)
    assert rec["sm_mhz"] == 1987.5 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"] and rec["samples"] == 4
    hot = sampler([row(1500, reasons=("Active", "Not Active", "Active", "Not Active"))])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert sampler([]) is None and sampler(["a, b"]) is None
