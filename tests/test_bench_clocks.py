"""The bench's clock record: only nvidia-smi samples that arrive inside the
timed region (plus one sampling period for the last) are summarised, and the
throttle reasons that the timing rules reject are reported."""

import bench


def _line(mhz, hw="Not Active", cap="Not Active"):
    return f"0, {mhz}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {cap}\n"


def _sampler(lines, region):
    s = bench.ClockSampler(0)
    s.lines = lines
    s.region = region
    return s


def test_samples_outside_the_region_are_dropped():
    lines = [(0.00, _line(600)), (0.05, _line(2070)), (0.07, _line(2060)),
             (0.09, _line(2070, cap="Active")), (0.30, _line(700))]
    out = _sampler(lines, (0.04, 0.08)).summary()
    assert out["window"] == "timed region"
    assert out["samples"] == 3                    # 0.05, 0.07 and 0.09 (ends within one period)
    assert out["sm_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_hw_slowdown_is_reported():
    lines = [(0.01, _line(1500, hw="Active")), (0.03, _line(1500))]
    out = _sampler(lines, (0.0, 0.03)).summary()
    assert "hw_slowdown" in out["reasons"]
    assert out["sm_mhz"] == 1500.0


def test_a_short_region_takes_the_nearest_sample():
    lines = [(0.0, _line(2070)), (1.0, _line(1000))]
    out = _sampler(lines, (0.10, 0.101)).summary()
    assert out["window"].startswith("nearest")
    assert out["samples"] == 1 and out["sm_mhz"] == 2070.0


def test_no_samples():
    out = _sampler([(0.0, "garbage\n")], (0.0, 1.0)).summary()
    assert out["reasons"] == ["unsampled"] and out["sm_mhz"] is None
