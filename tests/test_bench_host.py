"""Host logic of the bench: the clock record keeps only the nvidia-smi samples
that arrive inside the timed region (plus one sampling period for the last)
and reports the throttle reasons that the timing rules reject; the per-stage
report follows its stated algorithmic models."""

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


def test_stage_report_models_and_fractions():
    """The per-stage report: shares add to one, the reconstruction's bytes and
    the FFT's flops follow their stated models, and the fractions divide by
    the peaks given."""
    import math
    from paper_1604_08159_gb300 import workloads as W
    p = W.fujiwhara_1024().params
    ms = {"reconstruct": 0.5, "poisson": 1.0, "velocity": 0.05, "sgs": 0.25, "krylov": 2.5, "adapt": 0.6, "host": 0.1}
    r = bench.stage_report(ms, 5, p, 17000.0, 6800.0)
    N = float(p.NJ) ** 2
    assert abs(sum(r[k]["share"] for k in ms) - 1.0) < 1e-12
    assert abs(r["step_ms"] - sum(ms.values()) / 5) < 1e-12
    rec = r["reconstruct"]
    assert rec["algorithmic_bytes"] == 2 * 17 * N
    assert abs(rec["achieved"] - 2 * 17 * N / 0.1e-3 / 1e9) < 1e-6
    assert abs(rec["frac"] - rec["achieved"] / 6800.0) < 1e-12
    fft = r["poisson"]
    assert fft["algorithmic_flops"] == 5 * N * math.log2(N)
    assert abs(fft["frac"] - fft["achieved"] / bench.FP64_PEAK_GFLOPS) < 1e-12
    assert "frac" not in r["sgs"] and "frac" not in r["host"]
    mixed = W.RunParams(**{**p.as_dict(), "prec": W.PREC_MIXED})
    rm = bench.stage_report(ms, 5, mixed, 17000.0, 6800.0)
    assert rm["reconstruct"]["algorithmic_bytes"] == 2 * 9 * N     # 4-byte words
    assert "frac" not in rm["poisson"] and "frac" not in rm["krylov"]   # FP32 bulk: no FP64 model
