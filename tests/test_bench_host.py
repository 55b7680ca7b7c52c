"""bench.py's host-side pieces that need no GPU: the clock record (samples
stamped on arrival, only those in the sampled window kept, throttle reasons
collected) and the reference arm's JSON line (the CPU oracle on the same
workload and metric)."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(sm, mx, reasons=()):
    flags = ["Active" if nm in reasons else "Not Active"
             for nm in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")]
    return ", ".join(["0", str(sm), str(mx), "900.0", "0x0"] + flags) + "\n"


def test_clock_window_and_reasons():
    import bench

    lines = [(0.0, _line(1200, 2070)),            # before the window: idle
             (1.1, _line(2070, 2070)),
             (1.3, _line(2055, 2070, ["sw_power_cap"])),
             (1.5, _line(2070, 2070)),
             (2.9, _line(600, 2070, ["hw_slowdown"])),  # after the window
             (1.2, "garbage line\n")]
    out = bench.summarize_clocks(lines, 1.0, 2.0)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["window_s"] == pytest.approx(1.0)
    # no window: every parsable sample counts
    every = bench.summarize_clocks(lines, None, None)
    assert every["samples"] == 5 and every["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert "window_s" not in every
    # nothing sampled
    none = bench.summarize_clocks([], 1.0, 2.0)
    assert none["samples"] == 0 and none["sm_mhz"] is None


@pytest.mark.slow
def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600, check=True)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference"
    assert d["unit"] == "Newton steps/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["value"] > 0
    assert d["config"]["workload"] == "gn256"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
