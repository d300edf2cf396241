"""Host-side helpers of bench.py, on CPU: the byte models, the per-step
statistics and the guard that drops a measured DRAM figure once the
enumeration sources change.  No GPU is involved."""
import bench


def test_step_stats():
    st = bench.step_stats([82.0, 82.5, 83.0, 82.5])
    assert st["median"] == 82.5 and st["min"] == 82.0 and st["max"] == 83.0 and st["n"] == 4
    lo, hi = st["ci95_mean"]
    assert 82.0 <= lo <= 82.5 <= hi <= 83.0
    assert bench.step_stats([5.0])["ci95_mean"] == [5.0, 5.0]


def test_enumeration_byte_models():
    n, m = 1000, 8000
    # the enumeration pass: E+ once, 4 B per probe of the forward algorithm
    assert bench.enum_pass_bytes(n, m, 10_000) == 8 * (n + 1) + 4 * m + 40_000
    # the probes-made model adds the in-degrees, staged bounds and in-list entries
    assert bench.enum_streamed_bytes(n, m, 10_000) == 8 * (n + 1) + 4 * n + 4 * m + 8 * m + 8 * m + 40_000


def test_tr_step_byte_model():
    n, m, a_out, wf = 1000, 8000, 9000, 50_000
    A = 2 * m
    # read CSR, head degrees, write + read E+, forward probes, del flags, mask re-read, output
    want = (8 * n + 4 * A) + 4 * A + 2 * (8 * n + 4 * m) + 4 * wf + 2 * m + 4 * A + (8 * n + 4 * a_out)
    assert bench.tr_step_bytes(n, m, a_out, wf) == want


def test_streaming_byte_models():
    n, m, a_out = 1000, 8000, 9000
    A = 2 * m
    assert bench.byte_model(n, m, a_out, "compact_uniform") == 16 * (n + 1) + 4 * A + 4 * a_out
    assert bench.byte_model(n, m, a_out, "compact_spectral") == 16 * (n + 1) + 8 * A + 4 * a_out
    assert bench.byte_model(n, m, a_out, "nothing") is None


def test_measured_traffic_guarded_by_source_digest(monkeypatch):
    d = bench.sources_digest()
    assert len(d) == 64 and d == bench.sources_digest()
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, ("wl", "k"), (123, d))
    assert bench.measured_traffic("wl", "k") == 123
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, ("wl", "k"), (123, "0" * 64))
    assert bench.measured_traffic("wl", "k") is None
    assert bench.measured_traffic("no such workload", "k") is None


def test_streaming_rows_are_per_call():
    n, m, a_out, hbm = 1000, 8000, 9000, 6668.5
    # two profiled steps; the orientation is five launches per call
    kt = {"compact_orient": (4.0, 10), "tri_reverse_list": (6.0, 2), "compact_trmask": (0.0, 0)}
    rows = bench.streaming_rows(kt, 2, n, m, a_out, hbm)
    assert set(rows) == {"compact_orient", "tri_reverse_list"}
    o = rows["compact_orient"]
    assert o["ms"] == 2.0 and o["launches"] == 5.0
    b = bench.byte_model(n, m, a_out, "compact_orient")
    assert o["algorithmic_bytes"] == b
    assert abs(o["achieved"] - b / 2.0 / 1e6) < 1e-9 and abs(o["frac"] - b / 2.0 / 1e6 / hbm) < 1e-12
    assert rows["tri_reverse_list"]["ms"] == 3.0 and rows["tri_reverse_list"]["launches"] == 1.0
