"""Host logic of bench.py's opt-in sweep after the paper's benchmarking
algorithm (Algorithm 2): for every register size, `samples` runs, each of a
type drawn at random, in a seeded order.  No GPU involved."""
import collections
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_schedule_covers_every_size_with_samples_runs():
    s = bench.paper_sweep_schedule(28, 5, 1234)
    per_n = collections.Counter(n for n, _ in s)
    assert sorted(per_n) == list(range(1, 29))
    assert set(per_n.values()) == {5}
    # sizes in ascending order, as the algorithm's outer loop
    assert [n for n, _ in s] == sorted(n for n, _ in s)


def test_types_are_feasible_and_drawn_at_random():
    s = bench.paper_sweep_schedule(28, 40, 7)
    for n, t in s:
        assert t in bench.paper_types(n)
        if n < 11:
            assert t != "staged_c64"
    # every type shows up, and not in a fixed rotation
    assert set(t for _, t in s) == set(bench.PAPER_TYPES)
    assert s == bench.paper_sweep_schedule(28, 40, 7)
    assert s != bench.paper_sweep_schedule(28, 40, 8)


def test_summary_statistics():
    rows = [("a", 3, 0.001), ("a", 3, 0.004), ("a", 3, 0.002), ("b", 5, 0.010)]
    out = bench.summarize_sweep(rows)
    assert out["a"]["3"] == {"runs": 3, "mean_ms": 7.0 / 3.0, "median_ms": 2.0, "min_ms": 1.0}
    assert out["b"]["5"]["runs"] == 1 and out["b"]["5"]["min_ms"] == 10.0
