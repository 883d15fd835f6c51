"""Host arithmetic of bench.py, checked on the CPU: the algorithmic bytes per
cell-update agree with the per-stage array passes they are built from, the
profile record the roofline reads parses, and the issue roofline is withheld
when the kernel source no longer matches the profiled one."""
import re

import bench


def test_bytes_per_cell_update_equals_the_stage_passes():
    for precision, es in (("fp64", 8), ("fp32", 4), ("fp32dw", 4)):
        passes = sum(bench.STAGE_PASSES[precision])
        assert bench.bytes_per_cell_update(precision) == passes / 4 * bench.NF * es
    assert bench.bytes_per_cell_update("fp32dw") == 475.0
    assert bench.bytes_per_cell_update("fp64") == 800.0
    # the contract's figures: 16 RK4 passes (+ the Kahan read and write)
    assert bench.contract_bytes_per_cell_update("fp64") == 800.0
    assert bench.contract_bytes_per_cell_update("fp32dw") == 450.0


def test_profile_summary_parses():
    v = bench.profiled_values()
    assert v["traffic_bytes_per_launch"] > 0
    assert v["warp_instructions_per_launch"] > 0
    assert re.fullmatch(r"[0-9a-f]{16}", v["kernel_source_sha256_16"])
    assert re.fullmatch(r"[0-9a-f]{16}", bench.kernel_source_hash())


def test_issue_roofline_needs_the_profiled_source(monkeypatch):
    r32 = {"per_stage_ms": [0.3, 0.35, 0.35, 0.38]}
    clocks = {"sm_mhz": 2000.0}
    v = bench.profiled_values()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: v["kernel_source_sha256_16"])
    r = bench.issue_roofline(r32, clocks)
    t = sum(r32["per_stage_ms"]) / 4 * 1e-3
    assert r["peak"] == 152 * 4 * 2000.0e6
    assert abs(r["achieved"] - v["warp_instructions_per_launch"] / t) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.issue_roofline(r32, clocks) is None


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(4, 96 ** 3, 40, 10.0) == 4 * 96 ** 3 * 40 / 0.01


def test_nvml_summary_keeps_the_timed_window_only():
    # (host time, SM MHz, clock-event reason bits): the sample at t = 3.0 lies
    # after the window and carries hw_slowdown, which must not be reported
    samples = [(0.4, 1200, 0x1), (1.0, 2070, 0), (1.5, 2050, 0x4), (3.0, 1000, 0x8)]
    s = bench.NvmlSampler.summary(samples, [0.5, 2.0], 2070)
    assert s["samples_in_timed_region"] == 2
    assert s["sm_mhz"] == 2060.0 and s["sm_mhz_min"] == 2050 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]
    empty = bench.NvmlSampler.summary(samples, [None, None], None)
    assert empty["samples_in_timed_region"] == 0 and empty["sm_mhz"] is None


def test_nvml_sampler_without_a_driver_reports_nothing():
    s = bench.NvmlSampler(0)
    if s.lib is None:
        s.start()
        s.mark_start()
        s.mark_stop()
        assert s.stop() is None
