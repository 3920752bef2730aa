"""Host logic of bench.py that needs no GPU: the clock record's parsing (nvidia-smi CSV rows, the
loaded-sample filter and throttle reasons) and the number rounding of the JSON line."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_clock_rows_and_reasons():
    sys.path.insert(0, ROOT)
    import bench
    rows = bench.ClockSampler.parse([
        "0, 97, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 99, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 3, 345, 2070, 120.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    assert len(rows) == 3
    assert rows[1]["sm"] == 1980.0 and rows[1]["pcap"] == "Active"
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc, s.edges = None, []
    s.query = lambda: ""
    s.parse = bench.ClockSampler.parse
    # no samples and empty edge queries: no record
    assert s.stop() is None
    # the edge queries alone give a record (a timed region shorter than the sampling period)
    s.edges = ["0, 95, 2070, 2070, 800.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    rec = s.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["reasons"] == [] and "before" in rec["source"]


def test_significant_digits():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.sig(28703.259363912675) == 28700.0
    assert bench.sig(0.000123456, 2) == 0.00012
    assert bench.sig(None) is None and bench.sig(7) == 7
