"""The bench's committed records: the roofline denominator and the DRAM
traffic record must come from committed profiles, and the traffic must be
dropped once the scan kernel's sources differ from the ones captured."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_record_matches_current_kernel_sources():
    # the committed record was captured on the current sources
    t = bench.traffic_record()
    assert t is not None and 6.67e7 <= t <= 1e9   # at least the 2-bit words of a 266.7 Mbp pair


def test_traffic_record_dropped_when_sources_change(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "0000000000000000")
    assert bench.traffic_record() is None


def test_popc_rate_comes_from_the_committed_probe():
    # 16 POPC results per SM per clock, measured by the issue probe
    assert bench.popc_rate() == 16.0
