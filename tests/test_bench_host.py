"""Host logic of bench.py that needs no GPU: the clock sampler's summary (which
samples count, throttle reasons, the fallback when the timed steps are shorter
than the sampling interval) and the profile lookup behind roofline.traffic."""
import datetime
import hashlib
import os

import bench

FMT = "%Y/%m/%d %H:%M:%S.%f"


def _line(t, mhz, power_cap=False, thermal=False):
    ts = t.strftime(FMT)[:-3]
    cap = "Active" if power_cap else "Not Active"
    th = "Active" if thermal else "Not Active"
    return f"{ts}, 0, {mhz}, 2032, 900.0, 0x0, Not Active, {th}, Not Active, {cap}"


def _sampler(lines, t0=None, t1=None):
    c = bench.ClockSampler(0)
    c.lines = lines
    c.t0, c.t1 = t0, t1
    return c


def test_summary_keeps_the_timed_window():
    now = datetime.datetime(2026, 1, 2, 3, 4, 5)
    step = datetime.timedelta(milliseconds=20)
    lines = [_line(now + k * step, 1000 + k) for k in range(20)]
    # the timed steps cover samples 5 .. 9
    s = _sampler(lines, now + 5 * step, now + 9 * step).summary()
    assert s["samples"] == 5 and s["samples_total"] == 20
    assert s["sm_mhz"] == 1007.0          # median of 1005 .. 1009
    assert s["sm_max_mhz"] == 2032.0
    assert s["window"] == "timed steps" and s["reasons"] == []


def test_summary_reasons_only_inside_the_window():
    now = datetime.datetime(2026, 1, 2, 3, 4, 5)
    step = datetime.timedelta(milliseconds=20)
    lines = [_line(now + k * step, 2032, thermal=(k == 1), power_cap=(k == 6)) for k in range(10)]
    s = _sampler(lines, now + 5 * step, now + 8 * step).summary()
    assert s["reasons"] == ["sw_power_cap"]   # the thermal sample lies before the window


def test_summary_falls_back_to_the_last_second_before_a_short_window():
    now = datetime.datetime(2026, 1, 2, 3, 4, 5)
    step = datetime.timedelta(milliseconds=200)
    lines = [_line(now + k * step, 1900 + k) for k in range(5)]
    # a window between two samples: none inside, so the second before it counts
    t0 = now + 4 * step + datetime.timedelta(milliseconds=50)
    s = _sampler(lines, t0, t0 + datetime.timedelta(milliseconds=30)).summary()
    assert s["window"].startswith("warm-up") and s["samples"] == 5
    assert s["sm_mhz"] == 1902.0


def test_summary_without_timestamps_keeps_every_sample():
    lines = [f"n/a, 0, {1800 + k}, 2032, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
             for k in range(3)]
    s = _sampler(lines, datetime.datetime.now(), datetime.datetime.now()).summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 1801.0


def test_summary_of_no_output():
    s = _sampler([]).summary()
    assert s["sm_mhz"] is None and s["samples"] == 0


def test_traffic_record_needs_the_current_source():
    # the committed M2P summary names the current treecode.cu, so its DRAM bytes are used
    src = os.path.join(bench.ROOT, "paper_1309_4018_b300", "csrc", "treecode.cu")
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    txt = open(os.path.join(bench.ROOT, "profiles", "m2p_ly32_kernel_protein40k.md")).read()
    t = bench._traffic_record("treecode.cu", "m2p32")
    if f"source_sha256: {digest}" in txt:
        assert t is not None and t > 0
    else:
        assert t is None
    assert bench._traffic_record("treecode.cu", "no_such_kernel") is None
