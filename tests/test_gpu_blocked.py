"""Propagation-blocked Jacobi sweep (pr_tune.blocking) against the oracle:
the trajectory after k sweeps (FP64, the order of each vertex's sum varies
with the atomics, so agreement is to rounding), the converged result and
its stop rule, FP32, and at scale 24 in FP64 (a 134 MB vector, larger than
L2) a trajectory against the oracle's sweeps."""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import BOUND, D, graph, l1, top_order_matches

pytestmark = pytest.mark.gpu
BLOCKED = {"blocking": 1}


@pytest.fixture(scope="module")
def s16():
    n, src, dst = gen.rmat(16, 16, seed=1, dangling_frac=0.1)
    og = oracle.build_graph(n, src, dst)
    g = graph(n, src, dst)
    yield n, og, g
    g.close()


@pytest.mark.parametrize("use_graph", [True, False])
def test_blocked_trajectory_matches_oracle(s16, use_graph):
    n, og, g = s16
    for k in (1, 5, 17):
        x, r = g.solve(threshold=0.0, max_iter=k, tune=BLOCKED, use_graph=use_graph)
        ref = oracle.jacobi(og, D, tau=0.0, max_iter=k)
        assert r.iters == k
        assert l1(x, ref.x) <= 1e-13, k
        assert abs(r.sum_before_norm - ref.sum_before) <= 1e-13


def test_blocked_converges_like_jacobi(s16):
    n, og, g = s16
    star = oracle.fixed_point(og, D)
    x, r = g.solve(threshold=1e-10, tune=BLOCKED)
    ref = oracle.jacobi(og, D, tau=1e-10, max_iter=1000)
    assert r.status == 0 and abs(r.iters - ref.iters) <= 1
    assert l1(x, ref.x) <= 1e-10 and l1(x, star.x) <= BOUND
    assert top_order_matches(x.cpu().numpy(), star.x)
    x32, r32 = g.solve(threshold=1e-6, precision="fp32", tune=BLOCKED)
    assert r32.status == 0 and l1(x32, star.x) < 1e-5


def test_blocked_refuses_unsupported(s16):
    import paper_2203_09284_gb300 as fp
    n, og, g = s16
    for kw in ({"variant": "gs"}, {"precision": "fp32_dc"}, {"perforate_eps": 1e-6}):
        with pytest.raises(fp.PageRankError) as e:
            g.solve(tune=BLOCKED, **kw)
        assert e.value.status == fp.PR_ERR_UNSUPPORTED


def test_blocked_small_and_ragged_graphs():
    """Several bins with a ragged last bin, n = 1, no edges."""
    for n, src, dst in ((40000,) + gen.rmat(15, 8, seed=3)[1:],
                        (1, np.array([0], np.int32), np.array([0], np.int32)),
                        (7, np.zeros(0, np.int32), np.zeros(0, np.int32))):
        og = oracle.build_graph(n, src, dst)
        g = graph(n, src, dst)
        x, r = g.solve(threshold=0.0, max_iter=6, tune=BLOCKED)
        ref = oracle.jacobi(og, D, tau=0.0, max_iter=6)
        assert l1(x, ref.x) <= 1e-13, n
        g.close()


def test_blocked_scale24_fp64_beyond_l2():
    n, src, dst = gen.rmat(24, 16, seed=2)
    og = oracle.build_graph(n, src, dst)
    g = graph(n, src, dst)
    x, r = g.solve(threshold=0.0, max_iter=3, tune=BLOCKED)
    ref = oracle.jacobi(og, D, tau=0.0, max_iter=3)
    assert r.iters == 3
    assert l1(x, ref.x) <= 1e-13
    xp, _ = g.solve(threshold=0.0, max_iter=3)  # the in-list gather sweep
    assert l1(x, xp) <= 1e-13
    g.close()
