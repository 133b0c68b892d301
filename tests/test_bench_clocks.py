"""Host logic of the benchmark's clock record (no GPU): nvidia-smi samples are
kept only where their timestamps fall inside the timed region, throttle reasons
are collected from those samples, and a region that no sample falls into
reports the nearest sample with in_region false."""
import datetime
import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def stamp(t):
    return datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]


UUID = "GPU-00000000-1111-2222-3333-444444444444"


def sampler_with(rows, t0, t1, uuid=UUID):
    s = bench.ClockSampler(0, uuid=UUID)
    s.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    for t, sm, reasons in rows:
        flags = ["Active" if n in reasons else "Not Active"
                 for n in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")]
        s.f.write(", ".join([stamp(t), uuid, str(sm), "2070", "900.00", "0x0"] + flags) + "\n")
    s.f.flush()
    s.t0, s.t1 = t0, t1
    return s


def test_samples_outside_the_region_are_dropped():
    t0 = 1_800_000_000.0
    rows = [(t0 - 1.0, 1200, {"hw_slowdown"}),          # before the region: its slowdown must not count
            (t0 + 0.05, 2070, set()), (t0 + 0.10, 2060, {"sw_power_cap"}), (t0 + 0.15, 2070, set()),
            (t0 + 2.0, 900, {"sw_thermal_slowdown"})]   # after the region
    out = sampler_with(rows, t0, t0 + 0.2).summary()
    assert out["samples"] == 3 and out["in_region"] is True
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_region_without_samples_reports_the_nearest_one():
    t0 = 1_800_000_000.0
    rows = [(t0 - 0.5, 1980, set()), (t0 + 0.09, 2070, set()), (t0 + 3.0, 1500, {"hw_thermal_slowdown"})]
    out = sampler_with(rows, t0 + 0.05, t0 + 0.06).summary()
    assert out["in_region"] is False and out["samples"] == 1
    assert out["sm_mhz"] == 2070.0 and out["reasons"] == []


def test_malformed_lines_are_skipped_and_empty_log_gives_none():
    t0 = 1_800_000_000.0
    s = sampler_with([(t0 + 0.01, 2070, set())], t0, t0 + 0.1)
    s.f.write("garbage line\n, , ,\n")
    s.f.flush()
    out = s.summary()
    assert out["samples"] == 1
    assert sampler_with([], t0, t0 + 0.1).summary() is None


def test_samples_of_another_gpu_are_flagged():
    """The sampler asks nvidia-smi for the CUDA device's UUID; a sample that
    names another GPU (an index/ordinal mix-up) is reported, not hidden."""
    t0 = 1_800_000_000.0
    rows = [(t0 + 0.05, 2070, set())]
    assert sampler_with(rows, t0, t0 + 0.1).summary()["uuid_matches"] is True
    bad = sampler_with(rows, t0, t0 + 0.1, uuid="GPU-99999999-1111-2222-3333-444444444444").summary()
    assert bad["uuid_matches"] is False and bad["gpu_uuid"] == UUID
