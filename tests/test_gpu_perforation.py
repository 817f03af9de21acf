"""Loop-perforated Jacobi (the loop perforation the paper's related work and
conclusion name) on the GPU against the oracle's perforated iteration: the
same skip decisions (the count of gathered in-list entries is equal), the
same iterates to rounding, the stop rule's bound when only full sweeps stop,
and the unsupported combinations refused."""
import numpy as np
import torch
import pytest

import gen
import oracle
from gpu_util import BOUND, D, graph, l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def s16():
    n, src, dst = gen.rmat(16, 16, seed=1, dangling_frac=0.1)
    og = oracle.build_graph(n, src, dst)
    g = graph(n, src, dst)
    yield n, src, dst, og, g
    g.close()


@pytest.mark.parametrize("period", [0, 3])
def test_perforated_trajectory_matches_oracle(s16, period):
    n, src, dst, og, g = s16
    for k in range(1, 10):
        x, r = g.solve(threshold=0.0, max_iter=k, perforate_eps=3e-3, perforate_period=period)
        ref = oracle.perforated(og, D, eps=3e-3, period=period, tau=0.0, max_iter=k)
        assert r.iters == k
        assert r.gathered == ref.gathered, (k, r.gathered, ref.gathered)
        assert l1(x, ref.x) <= 1e-13, k
        assert abs(r.sum_before_norm - ref.sum_before) <= 1e-13, k
    assert ref.gathered < 9 * og.m  # vertices were skipped


def test_perforated_without_skips_is_jacobi(s16):
    n, src, dst, og, g = s16
    x, r = g.solve(threshold=1e-10, perforate_eps=1e-3, perforate_period=1)
    xj, rj = g.solve(threshold=1e-10)
    assert r.iters == rj.iters and r.gathered == rj.iters * og.m
    assert l1(x, xj) <= 1e-15


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_perforated_solve_reaches_the_bound(s16, precision):
    """period 4: the stop comes after a full sweep, so the stop rule's bound
    against the fixed point holds (FP64); period 0 is approximate: it gathers
    fewer in-list entries and is reported with its distance to x*."""
    n, src, dst, og, g = s16
    star = oracle.fixed_point(og, D)
    tau = 1e-10 if precision == "fp64" else 1e-6
    for eps in (1e-9, 1e-7):
        x, r = g.solve(threshold=tau, precision=precision, perforate_eps=eps,
                       perforate_period=4, max_iter=3000)
        assert r.status == 0 and (r.iters - 1) % 4 == 0
        bound = D / (1 - D) * tau + (0 if precision == "fp64" else 1e-5)
        assert l1(x, star.x) <= bound, (eps, l1(x, star.x))
        if precision == "fp64":
            ref = oracle.perforated(og, D, eps=eps, period=4, tau=tau, max_iter=3000)
            assert abs(r.iters - ref.iters) <= 4
        xa, ra = g.solve(threshold=tau, precision=precision, perforate_eps=eps,
                         perforate_period=0, max_iter=3000)
        assert ra.status == 0 and ra.gathered < ra.iters * og.m
        assert l1(xa, star.x) < 1e-3


def test_perforation_refuses_unsupported(s16):
    import paper_2203_09284_gb300 as fp
    n, src, dst, og, g = s16
    for kw in ({"variant": "gs"}, {"precision": "fp32_dc"}):
        with pytest.raises(fp.PageRankError) as e:
            g.solve(perforate_eps=1e-6, **kw)
        assert e.value.status == fp.PR_ERR_UNSUPPORTED
    with pytest.raises(fp.PageRankError) as e:
        g.solve(perforate_eps=1e-6, perforate_period=-1)
    assert e.value.status == fp.PR_ERR_INVALID_ARG


def test_perforation_degenerate_graphs():
    """n = 1, a graph without edges and an in-star: the perforated solve
    agrees with the dense solve of the Google matrix."""
    cases = [(1, [0], [0]), (5, [], []), (9, [1, 2, 3, 4, 5, 6, 7, 8], [0] * 8)]
    for n, s, t in cases:
        s = np.array(s, np.int32)
        t = np.array(t, np.int32)
        want = oracle.dense_pagerank(n, s, t, D)
        g = graph(n, s, t)
        for period in (0, 2):
            x, r = g.solve(threshold=1e-14, perforate_eps=1e-6, perforate_period=period,
                           max_iter=3000)
            assert r.status == 0, (n, period)
            err = np.abs(x.cpu().numpy() - want)
            if period:  # the stop follows a full sweep
                assert err.max() < 1e-12, (n, period)
            else:       # approximate: a kept vertex is off by about eps times its value
                assert (err <= 1e-5 * want).all(), (n, period)
        g.close()


def test_perforated_host_loop_matches_graph_loop(s16):
    """The host-driven loop (use_graph = 0) runs the same perforated sweeps."""
    n, src, dst, og, g = s16
    xa, ra = g.solve(threshold=1e-10, perforate_eps=1e-8, perforate_period=4)
    xb, rb = g.solve(threshold=1e-10, perforate_eps=1e-8, perforate_period=4, use_graph=False)
    assert ra.iters == rb.iters and ra.gathered == rb.gathered
    assert torch.equal(xa, xb)
