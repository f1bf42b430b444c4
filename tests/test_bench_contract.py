"""Host-side parts of the benchmark's JSON line: the DRAM traffic of the
pair kernel is reported only for the variant an ncu capture was taken on and
only while the kernel's sources are those it was taken on."""
import bench


def test_pair_traffic_only_for_the_captured_variant_and_sources(monkeypatch):
    captured = sorted(bench.PAIR_TRAFFIC["bytes"])
    assert captured, "no captured variant"
    for v in range(9):
        got = bench.pair_traffic(v)
        if v in captured:
            assert got == bench.PAIR_TRAFFIC["bytes"][v] and got > 0
        else:
            assert got is None
    # a changed kernel source: the stored figure no longer applies
    monkeypatch.setitem(bench.PAIR_TRAFFIC, "source_sha256", "0" * 64)
    assert all(bench.pair_traffic(v) is None for v in captured)
