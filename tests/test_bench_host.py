"""Host-side pieces of bench.py that need no GPU: the measured-traffic figure
is taken from the committed ncu summary only while the kernel sources hash to
the value that summary records."""
import bench


def test_source_hash_is_stable_and_hex():
    h = bench._source_hash()
    assert h == bench._source_hash()
    assert len(h) == 16 and int(h, 16) >= 0


def test_traffic_reported_only_for_the_profiled_sources(monkeypatch):
    t = bench._profiled_traffic()
    assert t is None or t > 0
    monkeypatch.setattr(bench, "_source_hash", lambda: "0" * 16)
    assert bench._profiled_traffic() is None


def test_peaks_read_from_measured_file():
    peak, kind = bench._peaks()
    assert peak > 1000 and kind in ("measured", "fallback")
