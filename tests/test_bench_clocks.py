"""The benchmark's clock record keeps the nvidia-smi samples that arrived
inside the timed region (or the first one after it), takes their median SM
clock and collects the throttle reasons they show."""
import bench


def line(sm, hw="Not Active", cap="Not Active"):
    return f"0, {sm}, 2070, 500.1, 0x0, {hw}, Not Active, Not Active, {cap}"


def test_summary_uses_samples_in_the_timed_region():
    c = bench.ClockSampler(0)
    c.lines = [(0.5, line(1000, hw="Active")), (1.1, line(2070)), (1.2, line(2040, cap="Active")),
               (1.3, line(2070)), (2.5, line(900))]
    c.t0, c.t1 = 1.0, 1.35
    s = c.summary()
    assert s["samples"] == 3 and s["in_timed_region"]
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]       # the hw_slowdown sample came before the region


def test_summary_falls_back_to_the_first_sample_after_a_short_region():
    c = bench.ClockSampler(0)
    c.lines = [(0.5, line(1000)), (1.4, line(2070, hw="Active")), (1.6, line(500))]
    c.t0, c.t1 = 1.0, 1.05
    s = c.summary()
    assert s["samples"] == 1 and not s["in_timed_region"]
    assert s["sm_mhz"] == 2070.0 and s["reasons"] == ["hw_slowdown"]


def test_summary_without_samples():
    c = bench.ClockSampler(0)
    assert c.summary() is None
