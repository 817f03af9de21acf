"""Input generator: determinism, dedup, dangling fix-up (no PageRank math)."""
import numpy as np

import gen


def test_rmat_is_deterministic_and_thread_independent():
    a = gen.rmat(14, 16, seed=3, threads=1)
    b = gen.rmat(14, 16, seed=3, threads=7)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    c = gen.rmat(14, 16, seed=4)
    assert not np.array_equal(a[1][:100], c[1][:100])


def test_rmat_dedup_and_ranges():
    n, s, d = gen.rmat(12, 16, seed=2)
    assert s.min() >= 0 and s.max() < n and d.min() >= 0 and d.max() < n
    assert not (s == d).any()
    key = s.astype(np.int64) * n + d
    assert len(np.unique(key)) == len(key)
    # skewed degrees, as R-MAT should be
    deg = np.bincount(d, minlength=n)
    assert deg.max() > 20 * deg.mean()


def test_dangling_fixup_exact_fraction():
    for scale in (10, 13):
        n, s, d = gen.rmat(scale, 16, seed=1, dangling_frac=0.10)
        out = np.bincount(s, minlength=n)
        assert (out == 0).sum() == round(0.10 * n)
        key = s.astype(np.int64) * n + d
        assert len(np.unique(key)) == len(key) and not (s == d).any()


def test_workload_draws():
    w = gen.edge_weights(1000, 1)
    assert w.dtype == np.float32 and (w > 0).all() and (w <= 1).all()
    t, c = gen.loss_targets(100, 5000, 2)
    assert len(np.unique(t)) == 100 and (np.abs(c) < 1).all()
    shapes = gen.multi_graph_shapes(64, 3)
    assert all(10 <= s <= 18 and 8 <= e <= 32 for s, e in shapes)
    assert len({s for s, _ in shapes}) > 5
