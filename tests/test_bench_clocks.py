"""The benchmark's clock record (`bench.ClockSampler`): median SM clock under
load, the maximum, and the throttle reasons seen active in any sample, parsed
from nvidia-smi's CSV (no GPU needed: a stand-in process and a written file)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")
    s = bench.ClockSampler(0)
    s.path = str(p)
    s.fh = open(p, "a")
    s.proc = _Done()
    return s


def test_median_max_and_no_reasons(tmp_path):
    rows = ["0, %d, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active" % mhz
            for mhz in (2070, 2070, 1980, 2070, 2055)]
    out = _sampler(tmp_path, rows).stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 5
    assert out["reasons"] == []


def test_reasons_seen_in_any_sample(tmp_path):
    rows = ["0, 2070, 2070, 1300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1800, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1500, 2070, 1400.0, 0x8, Active, Not Active, Active, Not Active",
            "garbage line",
            "0, [N/A], 2070, 1400.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    out = _sampler(tmp_path, rows).stop()
    assert out["samples"] == 3 and out["sm_mhz"] == 1800.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_no_sampler_is_reported():
    out = bench.ClockSampler(0).stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]
