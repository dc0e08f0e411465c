"""Host-side helpers of bench.py: the clock window summary (only samples inside
a line's timed window count, throttle reasons are collected, no samples is
reported as such), the sort-bandwidth line, and the DRAM traffic that is
reported only while the kernel sources hash to the recorded digest."""
import datetime
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _row(ts, sm, smax, reasons=("Not Active",) * 4):
    stamp = datetime.datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([stamp, "0", str(sm), str(smax), "900.00", "0x0"] + list(reasons))


def test_clock_summary_keeps_only_the_window():
    c = bench.ClockSampler(0)
    t0 = 1_700_000_000.0
    c.windows["a"] = [t0, t0 + 2.0]
    c.lines = [_row(t0 - 5, 1000, 2070),            # before the window
               _row(t0 + 0.5, 2070, 2070),
               _row(t0 + 1.0, 2040, 2070, ("Not Active", "Not Active", "Not Active", "Active")),
               _row(t0 + 1.5, 2070, 2070),
               _row(t0 + 9, 500, 2070, ("Active",) * 4)]  # after it
    s = c.summary("a")
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_without_samples():
    c = bench.ClockSampler(0)
    c.windows["a"] = [0.0, 1.0]
    c.lines = ["garbage", ""]
    assert c.summary("a") == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}


def test_sort_line_bytes_and_rate():
    line = bench._sort_line({"sort": 2.0}, points=1000, digits=20000)
    assert line["bytes"] == 64 * 1000 + 8 * 20000
    assert line["achieved"] == pytest.approx(line["bytes"] / 2e-3 / 1e9)
    assert line["frac"] == pytest.approx(line["achieved"] / line["peak"])
    assert bench._sort_line({}, 1, 1) is None


def test_verify_traffic_follows_the_source_digest(tmp_path, monkeypatch):
    import hashlib

    # a copy of the listed sources, with the recorded digest set to the copy's
    src = os.path.join(ROOT, "paper_2501_03245_gb300", "csrc")
    dst = tmp_path / "paper_2501_03245_gb300" / "csrc"
    dst.mkdir(parents=True)
    h = hashlib.sha256()
    for f in bench.VERIFY_TRAFFIC["sources"]:
        shutil.copy(os.path.join(src, f), dst / f)
        h.update((dst / f).read_bytes())
    rec = dict(bench.VERIFY_TRAFFIC, digest=h.hexdigest()[:16], bytes=123456789)
    monkeypatch.setattr(bench, "VERIFY_TRAFFIC", rec)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    n = rec["batch"]
    assert bench.verify_traffic(n) == 123456789
    assert bench.verify_traffic(n // 2) is None  # another batch size
    with open(dst / rec["sources"][0], "a") as fh:  # one source changed by a byte
        fh.write("\n")
    assert bench.verify_traffic(n) is None
