"""Host-side logic of bench.py that needs no GPU: the clock sampler (against a stand-in for nvidia-smi
that prints the same CSV lines) and the throttle-reason decoding."""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

FAKE = ("import sys, time\n"
        "for k in range(200):\n"
        "    mask = '0x0000000000000004' if k == 3 else '0x0000000000000001' if k == 0 else '0x0000000000000000'\n"
        "    print(f'{2070 if k else 1980}, 2070, {300 + k}.5, {mask}', flush=True)\n"
        "    time.sleep(0.02)\n")


def test_clock_sampler_is_live_at_start_and_decodes_reasons():
    s = bench.ClockSampler(0, cmd=[sys.executable, "-c", FAKE])
    t0 = time.perf_counter()
    s.start()
    assert s.samples, "start() returns once the first sample has arrived"
    assert time.perf_counter() - t0 < 3.0
    time.sleep(0.3)
    out = s.stop()
    assert out["samples"] >= 5
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    # gpu_idle (0x1) is dropped, sw_power_cap (0x4) is kept
    assert out["reasons"] == ["sw_power_cap"]
    assert out["power_w_max"] > 300.0


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0, cmd=["/nonexistent/nvidia-smi"])
    s.start()
    out = s.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_reason_mask_decoding():
    assert bench._reasons(0x8 | 0x20 | 0x40) == ["hw_slowdown", "sw_thermal_slowdown", "hw_thermal_slowdown"]
    assert bench._reasons(0) == []
