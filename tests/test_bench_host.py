"""Host-side parts of bench.py that need no GPU."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_cpu_batch_sample_runs_the_oracle_on_host_cores():
    import bench
    import synth
    g, _ = synth.config1()
    queries = [(0, 1023), (5, 900), (31, 992), (100, 700), (64, 1000), (2, 513)]
    out = bench.cpu_batch_sample(g, queries, every=2, budget=0)
    assert out["kind"] == "oracle" and out["unit"] == "queries/s" and out["value"] > 0
    assert 1 <= out["cores"] <= 3
    assert "3 of the 6 queries (1 in 2)" in out["sample"] and "0 over budget" in out["sample"]


def test_cpu_batch_sample_reports_queries_over_budget():
    import bench
    import synth
    g, _ = synth.config1()
    out = bench.cpu_batch_sample(g, [(0, 1023), (0, 1023)], every=1, budget=50)
    assert "2 over budget" in out["sample"]


def test_traffic_digest_covers_the_kernel_sources_and_launch_options():
    import bench
    a = bench.kernel_source_digest((1024, 8, 32, 1))
    assert len(a) == 16 and a == bench.kernel_source_digest((1024, 8, 32, 1))
    assert a != bench.kernel_source_digest((512, 8, 32, 1))
    assert all(os.path.exists(os.path.join(ROOT, f)) for f in bench.KERNEL_SOURCES)
    assert all(len(k) == 16 and isinstance(v, int) and v > 0 for k, v in bench.TRAFFIC.items())


def test_kernel_digest_ignores_comments_only():
    import bench
    a = "int f(int x) {  // add one\n  return x + 1; /* done */\n}\n"
    b = "/* header */\nint f(int x) {\n  return x + 1;\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench.strip_comments(a) == bench.strip_comments(b) != bench.strip_comments(c)


def test_oracle_count_bytes_of_the_headline_query():
    """The per-unit figures applied to the committed oracle counters of the
    256x256 d=3 query (written by tests/golden/make_golden.py)."""
    import bench
    fx = bench.fixture_stats()
    d = 3
    expect = (fx["extracted"] * 36 + fx["candidates"] * 28 + fx["comparisons"] * 12 + fx["inserted"] * 36
              + 4 * (fx["pruned_open"] + fx["pruned_open_goal"] + fx["pruned_closed"] + fx["pruned_p"]))
    assert bench.oracle_count_bytes(fx, d) == expect
    assert 7.0e11 < expect < 7.5e11


def test_grid_distance_estimates_query_cost():
    import bench
    import synth
    g, _ = synth.config1()
    assert bench.grid_distance(g, [(0, 1023), (0, 33), (5, 5)]) == [31, 1, 0]
    r, _ = synth.time_route(1, 3, 4, 6, 2)
    assert bench.grid_distance(r, [(0, r.n - 1)]) == [1]
