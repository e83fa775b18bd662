"""Host-side logic of the benchmark on CPU: the clock summary keeps only the nvidia-smi samples
taken inside the timed region and reports the throttle reasons they saw, and the reference arm's
per-step window shrinks for long runs but never below 16 rows."""
import datetime
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Done:
    """Stands in for the finished nvidia-smi process."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _row(t, index, sm, power_cap):
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    cap = "Active" if power_cap else "Not Active"
    return f"{stamp}, {index}, {sm}, 2070, 950.25, 0x0000000000000000, Not Active, Not Active, Not Active, {cap}\n"


def test_clock_summary_keeps_the_samples_of_the_timed_region(tmp_path):
    t0 = time.time()
    path = tmp_path / "clocks.csv"
    path.write_text(_row(t0 - 0.4, 0, 1200, False) +   # before the region (idle clocks)
                    _row(t0 + 0.1, 0, 2070, False) +
                    _row(t0 + 0.3, 1, 900, True) +     # another GPU of the machine
                    _row(t0 + 0.5, 0, 2040, True) +
                    _row(t0 + 1.5, 0, 1100, False))    # after the region
    s = bench._clock_summary(_Done(), str(path), 0, t0, t0 + 0.6)
    assert s["samples"] == 2 and s["samples_in_timed_region"] == 2
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert not path.exists()


def test_clock_summary_falls_back_to_all_samples(tmp_path):
    t0 = time.time()
    path = tmp_path / "clocks.csv"
    path.write_text(_row(t0 - 1.0, 0, 2070, False))
    s = bench._clock_summary(_Done(), str(path), 0, t0, t0 + 0.02)
    assert s["samples"] == 1 and s["samples_in_timed_region"] == 0 and s["sm_mhz"] == 2070.0


def test_reference_window_is_bounded():
    x0, y0, w, h = bench.REF_WINDOW
    assert bench.ref_window(3) == bench.REF_WINDOW
    assert bench.ref_window(200) == bench.REF_WINDOW
    rows = [bench.ref_window(k)[3] for k in (201, 400, 600, 10**6)]
    assert rows == sorted(rows, reverse=True) and rows[0] < h and rows[-1] == 16
    assert all(bench.ref_window(k)[:3] == (x0, y0, w) for k in (1, 600, 10**6))


def test_captured_counters_only_describe_the_captured_build():
    """ncu counters attach to the bench line only for the kernel sources and the tile /
    samples-per-group they were captured with."""
    saved = dict(bench.CAPTURED)
    try:
        bench.CAPTURED.update(sources=bench.kernel_sources_sha(), tile=8, spt=2,
                              kernels={"raster_bwd_persistent": {"dram_bytes": 1.0, "pipes_pct": {}}})
        assert bench.captured_counters("raster_bwd_persistent", 8, 2) == {"dram_bytes": 1.0, "pipes_pct": {}}
        assert bench.captured_counters("raster_bwd_persistent", 8, 1) is None
        assert bench.captured_counters("raster_fwd_persistent", 8, 2) is None
        bench.CAPTURED["sources"] = "0" * 16
        assert bench.captured_counters("raster_bwd_persistent", 8, 2) is None
    finally:
        bench.CAPTURED.clear()
        bench.CAPTURED.update(saved)
