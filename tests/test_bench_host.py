"""Host logic of bench.py (no GPU): the clock-sample summary of the timed window
and the source hash that guards the captured DRAM-traffic figure."""
import datetime
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(t, uuid="GPU-abc", sm=2070, mx=2070, reasons=("Not Active",) * 4):
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([stamp, uuid, str(sm), str(mx), "900.0", "0x0"] + list(reasons)) + "\n"


def test_clock_window_keeps_samples_inside():
    t0 = 1_800_000_000.0
    lines = [_line(t0 - 0.5, sm=1000), _line(t0 + 0.1, sm=2000), _line(t0 + 0.2, sm=2060),
             _line(t0 + 0.3, sm=2070), _line(t0 + 2.0, sm=500)]
    out = bench.summarize_clocks(lines, "abc", t0, t0 + 0.35)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2060
    assert out["sm_max_mhz"] == 2070
    assert out["reasons"] == []
    assert out["window_ms"] == 350.0


def test_clock_window_reasons_and_uuid_filter():
    t0 = 1_800_000_000.0
    hot = ("Not Active", "Active", "Not Active", "Active")
    lines = [_line(t0 + 0.1, reasons=hot), _line(t0 + 0.2, uuid="GPU-other", sm=10)]
    out = bench.summarize_clocks(lines, "abc", t0, t0 + 0.5)
    assert out["samples"] == 1
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_window_shorter_than_period_takes_next_sample():
    t0 = 1_800_000_000.0
    lines = [_line(t0 - 0.05, sm=1), _line(t0 + 0.12, sm=2070), _line(t0 + 0.22, sm=3)]
    out = bench.summarize_clocks(lines, None, t0, t0 + 0.07)
    assert out["samples"] == 1 and out["sm_mhz"] == 2070
    assert bench.summarize_clocks(lines[:1], None, t0, t0 + 0.07) is None


def test_source_hash_marker_covers_the_prefix():
    d = os.path.join(ROOT, "paper_1505_00354_gb300", "csrc")
    fft = open(os.path.join(d, "fft.cu"), "rb").read()
    hdr = open(os.path.join(d, "gbdlt_internal.cuh"), "rb").read()
    cut = hdr.find(b"\n// plan\n")
    assert cut > 0
    want = hashlib.sha256(fft + hdr[:cut]).hexdigest()[:16]
    assert bench.src_hash(("fft.cu", ("gbdlt_internal.cuh", "// plan"))) == want
    # the traffic figure is reported only while this hash matches the capture's
    t = bench.TRAFFIC["fft_cols"]
    assert len(t["src"]) == 16
