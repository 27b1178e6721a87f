"""The seeded generators draw what their docstrings promise (no GPU)."""
import numpy as np

from paper_1706_06940_gb300 import workloads as W


def test_uniform_array_range_and_determinism():
    a = W.uniform_array(100_000, 1)
    assert a.dtype == np.int32 and a.min() >= 0
    assert np.array_equal(a, W.uniform_array(100_000, 1))
    assert not np.array_equal(a, W.uniform_array(100_000, 2))


def test_uniform_queries_ordered_and_in_range():
    l, r = W.uniform_queries(1000, 50_000, 3)
    assert (l <= r).all() and l.min() >= 0 and r.max() < 1000


def test_paper_permutation_is_a_permutation():
    a = W.paper_permutation(100_000, 4)
    assert np.array_equal(np.sort(a), np.arange(1, 100_001, dtype=np.int32))
    assert (a != np.arange(1, 100_001)).mean() > 0.3     # n/2 swaps move ~60% of cells


def test_log_width_queries():
    n = 100_000
    l, r = W.log_width_queries(n, 200_000, 5, 1, 10_000)
    w = r - l + 1
    assert (l >= 0).all() and (r < n).all() and w.min() >= 1 and w.max() <= 10_000
    assert abs(np.mean(w < 1024) - np.log(1024) / np.log(10_000)) < 0.01


def test_served_sizes_sum_and_clamp():
    s = W.served_array_sizes(64, 4_000_000_000, 6)
    assert s.sum() == 4_000_000_000 and s.max() <= 2e8 + 64 and s.min() > 0
