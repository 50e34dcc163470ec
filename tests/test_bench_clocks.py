"""The bench's clock record on the CPU, against a stand-in nvidia-smi.

bench.ClockSampler runs `nvidia-smi --query-gpu=... -lms 200` beside the
timed region and turns its rows into the line's `clocks` entry: the median
SM clock under load, the maximum clock, and the throttle reasons that a run
must not have seen.  A stand-in script on PATH prints rows like the real
tool, so the parsing, the wait for the first sample and the reasons are
checked without a GPU.
"""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

# index, clocks.sm, clocks.max.sm, power.draw, active, hw_slowdown,
# hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
ROWS = {
    "clean": ["0, 2070, 2070, 650.1, 0x0, Not Active, Not Active, Not Active, Not Active"] * 3,
    "power": ["0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
              "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
              "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active"],
    "thermal": ["0, 1500, 2070, 900.0, 0x20, Not Active, Active, Not Active, Not Active"] * 3,
    # an idle row (clock far below the others) is not counted as under load
    "idle": ["0, 345, 2070, 90.0, 0x1, Not Active, Not Active, Not Active, Not Active",
             "0, 2070, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2055, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active"],
}


def fake_smi(tmp_path, rows, delay=0.0):
    """An executable named nvidia-smi that waits `delay` s (start-up), then
    prints one row every 50 ms, cycling through `rows`, until terminated."""
    script = tmp_path / "nvidia-smi"
    body = "\n".join([
        f"#!{sys.executable}",
        "import sys, time",
        f"time.sleep({delay})",
        f"rows = {rows!r}",
        "k = 0",
        "while True:",
        "    print(rows[k % len(rows)], flush=True)",
        "    k += 1",
        "    time.sleep(0.05)",
    ])
    script.write_text(body + "\n")
    script.chmod(script.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


@pytest.mark.parametrize("case,sm,reasons", [
    ("clean", 2070.0, []),
    ("power", 2070.0, ["sw_power_cap"]),
    ("thermal", 1500.0, ["hw_thermal_slowdown"]),
    ("idle", 2062.5, []),
])
def test_clock_record(tmp_path, monkeypatch, case, sm, reasons):
    monkeypatch.setenv("PATH", fake_smi(tmp_path, ROWS[case]) + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(0)
    time.sleep(0.3)
    rec = c.stop()
    assert rec["sm_mhz"] == sm
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == reasons
    assert rec["samples"] >= 3


def test_first_sample_before_the_timed_region(tmp_path, monkeypatch):
    """The sampler returns only once the tool has printed its first row (its
    start-up would otherwise fall inside a short timed region), and that row
    is kept in the record."""
    monkeypatch.setenv("PATH", fake_smi(tmp_path, ROWS["clean"], delay=0.4) + os.pathsep + os.environ["PATH"])
    t0 = time.monotonic()
    c = bench.ClockSampler(0)
    waited = time.monotonic() - t0
    assert waited >= 0.35
    assert len(c.first) == 1
    rec = c.stop()  # stopped at once: the first row alone
    assert rec["samples"] >= 1 and rec["sm_mhz"] == 2070.0


def test_no_tool(tmp_path, monkeypatch):
    """Without nvidia-smi the record says so instead of failing the run."""
    monkeypatch.setenv("PATH", str(tmp_path))
    rec = bench.ClockSampler(0).stop()
    assert rec["sm_mhz"] is None
    assert rec["reasons"] == ["nvidia-smi unavailable"]
