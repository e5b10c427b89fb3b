"""Host-side logic of bench.py (CPU): the per-pair work counts behind the
roofline figures and the clock-record summary that decides whether a timed
run is kept."""
import bench


def test_fp32_flops_per_pair():
    # forward N^2 + 4N + 7, backward 2N^2 + 7N + 13 (counted in the docstring)
    assert bench.flops_per_pair(6) == (67, 127)
    assert bench.flops_per_pair(10) == (147, 283)


def test_tensor_core_flops_per_pair():
    # N = 6: F = 21 + 6 + 1 = 28 lifted features, K padded to 32; backward
    # S: 3 products x 2 x 32; E Psi: 2 products x 2 x (3 x 32)
    assert bench.tc_flops_per_pair(6) == (56, 112, 192, 192 + 384)
    # N = 10: F = 55 + 10 + 1 = 66, K padded to 80
    assert bench.tc_flops_per_pair(10) == (132, 264, 480, 480 + 960)
    # F a multiple of 16: no padding (N = 1: F = 3 -> 16)
    assert bench.tc_flops_per_pair(1)[2] == 6 * 16


def test_fp32_peak():
    # 152 SMs x 128 lanes x 2 flops x 2070 MHz
    assert abs(bench.fp32_peak_tflops(2070.0) - 80.55) < 0.01


def _line(mhz, mx, reasons):
    flags = ["Active" if r else "Not Active" for r in reasons]
    return f"0, {mhz}, {mx}, 900.0, 0x0, " + ", ".join(flags)


def test_clock_summary_median_max_and_reasons():
    s = bench.ClockSampler(0)
    s.lines = [_line(2070, 2070, (0, 0, 0, 0)), _line(1980, 2070, (0, 0, 0, 1)),
               _line(2055, 2070, (0, 0, 0, 0)), "garbage line", ""]
    out = s.summary()
    assert out["sm_mhz"] == 2055.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_throttling():
    s = bench.ClockSampler(0)
    s.lines = [_line(1500, 2070, (1, 1, 0, 0)), _line(1600, 2070, (0, 0, 1, 0))]
    assert s.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0)
    out = s.summary()
    assert out["sm_mhz"] is None and out["samples"] == 0 and out["reasons"] == []


def test_oracle_thread_control_for_the_cpu_baseline(oracle):
    # the baseline reports the oracle's own thread count and times one core
    n = oracle.threads()
    assert n >= 1
    try:
        oracle.set_threads(1)
        assert oracle.threads() == 1
    finally:
        oracle.set_threads(n)
    assert oracle.threads() == n
