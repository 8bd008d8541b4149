"""The bench's reading of the nvidia-smi clock samples taken during the timed
region (host only, from recorded sample lines)."""
import bench


def _summary(lines):
    c = bench.ClockSampler(0)
    c.out.write("\n".join(lines) + "\n")
    return c.summary()


def test_median_clock_max_and_reasons():
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1965, 2070, 1380.5, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = _summary(rows)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_thermal_and_hardware_slowdowns_are_reported():
    rows = ["0, 1500, 2070, 1000, 0x48, Active, Not Active, Active, Not Active"]
    assert _summary(rows)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_unavailable_fields_and_no_samples():
    s = _summary(["0, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]"])
    assert s["sm_mhz"] is None and s["sm_max_mhz"] is None and s["samples"] == 1
    s = _summary([])
    assert s["samples"] == 0 and s["reasons"] == ["nvidia-smi unavailable"]
