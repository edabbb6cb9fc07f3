"""Host-side pieces of the benchmark, on the CPU: the committed DRAM-traffic
record is used only while the kernel's sources still hash to the captured
value, and the clock sampler's parser reports the median SM clock and every
throttle reason it saw."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_committed_leaf_traffic_matches_current_sources():
    files = ["minplus.cu", "minplus_tile.cuh"]
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["minplus16_leaf_n4096"]
    if rec["source_sha"] == bench.source_sha(files):
        assert bench.ncu_traffic(files, "minplus16_leaf_n4096") == rec["dram_bytes_per_launch"]
    else:  # the leaf changed after the capture: the bench must report no traffic
        assert bench.ncu_traffic(files, "minplus16_leaf_n4096") is None


def test_traffic_dropped_when_sources_change(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1911_05328_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_text("kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.source_sha(["k.cu"])
    (tmp_path / "profiles" / "traffic.json").write_text(
        json.dumps({"k_case": {"source_sha": sha, "dram_bytes_per_launch": 1234}}))
    assert bench.ncu_traffic(["k.cu"], "k_case") == 1234
    (csrc / "k.cu").write_text("kernel v2")
    assert bench.ncu_traffic(["k.cu"], "k_case") is None
    assert bench.ncu_traffic(["k.cu"], "missing_case") is None


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_parser(tmp_path):
    path = tmp_path / "clocks.csv"
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
        "0, 1500, 2070, 1200.0, 0x8, Active, Not Active, Not Active, Not Active",
    ]
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.path = str(path)
    s.f = open(s.path, "w")
    s.f.write("\n".join(rows) + "\n")
    s.p = _Done()
    out = s.stop()
    assert out["samples"] == 4
    assert out["sm_mhz"] == 2025.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert not os.path.exists(s.path)


def test_bench_row_sample_matches_the_tests_row_sample():
    """The benchmark measures its errors on the same rows as the tests: an
    even spread plus the quadrant edges of four halvings."""
    import numpy as np

    import oracle

    for m in (256, 8192, 12288, 16384):
        np.testing.assert_array_equal(bench.sample_rows(m), oracle.sample_rows(m))
        r = bench.sample_rows(m)
        assert r[0] == 0 and r[-1] == m - 1 and np.all(np.diff(r) > 0)
        assert {m // 2 - 1, m // 2, m // 16 - 1, m // 16}.issubset(set(r.tolist()))


def test_error_book_keeps_each_input_set():
    """Sampled-row errors are computed after the GPU phase from the inputs
    registered for each set, even when the caller reuses its variable names
    for the next workload (the sets must hold their own arrays)."""
    import numpy as np

    import oracle

    book = bench.ErrBook()
    rng = np.random.default_rng(0)
    A = rng.uniform(-1, 1, (8, 5))
    B = rng.uniform(-1, 1, (5, 6))
    rows = np.array([0, 3, 7])
    book.add_set("first", lambda A=A, B=B: (A, B), rows)
    rec1 = {}
    book.add("first", rec1, "error", (A @ B)[rows] * (1 + 1e-9))
    A = rng.uniform(-1, 1, (4, 9))  # the next workload reuses the names
    B = rng.uniform(-1, 1, (9, 3))
    book.add_set("second", lambda A=A, B=B: (A, B), np.arange(4))
    rec2 = {}
    book.add("second", rec2, "error", A @ B)
    Ai = rng.integers(0, 1001, (6, 6)).astype(np.int32)
    book.add_set("mp", lambda A=Ai: (A, A), np.arange(6), kind="minplus")
    rec3 = {}
    book.add("mp", rec3, "exact", oracle.mm_minplus(Ai, Ai))
    book.resolve(oracle)
    assert abs(rec1["error"] - 1e-9) < 1e-12
    assert rec2["error"] < 1e-14
    assert rec3["exact"] is True
