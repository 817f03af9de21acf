"""The launch-parameter search on the GPU: the chosen parameters are the
fastest measured, cached, and change no result."""
import pytest
import torch

import gen
from gpu_util import graph, l1

pytestmark = pytest.mark.gpu


def test_autotune_choice_cache_and_results(tmp_path):
    from paper_2203_09284_gb300 import tune
    n, src, dst = gen.rmat(16, 16, seed=7, dangling_frac=0.1)
    g = graph(n, src, dst)
    cache = str(tmp_path / "tune.json")
    cands = tune.DEFAULT_CANDIDATES[:6]
    best, rep = tune.autotune(g, precision="fp64", candidates=cands, sweeps=4, cache=cache)
    assert not rep["cached"] and best in cands
    t = {int(k): v for k, v in rep["times_ms"].items()}
    assert t[cands.index(best)] == min(t.values())
    again, rep2 = tune.autotune(g, precision="fp64", candidates=cands, cache=cache)
    assert rep2["cached"] and again == best
    x0, _ = g.solve(threshold=0.0, max_iter=9)
    x1, _ = g.solve(threshold=0.0, max_iter=9, tune=best)
    assert l1(x0, x1) <= 1e-13  # same iterates up to summation order
    g.close()


def test_autotune_multi_family():
    import paper_2203_09284_gb300 as fp
    from paper_2203_09284_gb300 import tune
    gs = [graph(*gen.rmat(sc, 8, seed=sc)) for sc in (10, 12, 13)]
    best, times = tune.autotune_multi(gs, precision="fp32", candidates=tune.DEFAULT_CANDIDATES[:4],
                                      sweeps=3)
    assert best in tune.DEFAULT_CANDIDATES[:4] and len(times) == 4
    xa, _ = fp.solve_multi(gs, threshold=1e-10)
    xb, _ = fp.solve_multi(gs, threshold=1e-10, tune=best)
    for a, b in zip(xa, xb):
        assert l1(a, b) <= 1e-11
    for g in gs:
        g.close()
