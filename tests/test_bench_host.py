"""Host-side helpers of bench.py.  The clock record: median SM clock under load, the
maximum clock and every throttle reason seen while the timed region ran (a run that saw
a hardware or thermal slowdown is rejected, so the reasons must not be lost).  The extra
sections: a failing one is recorded in the line instead of losing the line."""
import bench


def test_clock_summary_reports_median_max_and_every_reason_seen():
    lines = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1980, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "[N/A]\n",                                                   # a malformed row is skipped
        "0, 1200, 2070, 1390.0, 0x0000000000000008, Active, Not Active, Not Active, Active\n",
    ]
    c = bench.summarize_clock_samples(lines)
    assert c["samples"] == 3
    assert c["sm_mhz"] == 1980.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_summary_of_a_quiet_run_and_of_no_samples():
    quiet = ["0, 2070, 2070, 700.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"] * 5
    c = bench.summarize_clock_samples(quiet)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}
    empty = bench.summarize_clock_samples([])
    assert empty["sm_mhz"] is None and empty["samples"] == 0


def test_a_failing_extra_section_is_recorded_not_raised():
    def boom(x):
        raise RuntimeError(f"device said no ({x})")
    assert bench.guarded(lambda a, b=0: a + b, 2, b=3) == 5
    assert bench.guarded(boom, 7) == {"error": "RuntimeError: device said no (7)"}
