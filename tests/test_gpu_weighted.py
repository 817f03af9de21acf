"""Weighted PageRank (P_uv = w_uv / s_u per edge) on the GPU vs the oracle's
row-normalised sweep, for every sweep and precision."""
import numpy as np
import pytest
import torch

import gen
import oracle
from gpu_util import BOUND, D, graph, l1

pytestmark = pytest.mark.gpu

DC_BOUND = 1e-10 / (1 - D)


@pytest.fixture(scope="module")
def wgraph():
    n, src, dst = gen.rmat(14, 12, seed=31, dangling_frac=0.08)
    w = gen.edge_weights(len(src), seed=31)
    og = oracle.build_graph(n, src, dst)
    _, _, csc_p = oracle.row_normalize(og, w)
    g = graph(n, src, dst, w=w)
    star = oracle.fixed_point(og, D, csc_p=csc_p)
    yield n, og, csc_p, g, star
    g.close()


@pytest.mark.parametrize("k", [1, 4, 13])
def test_weighted_jacobi_fp64_trajectory(wgraph, k):
    n, og, csc_p, g, star = wgraph
    x, r = g.solve(threshold=0.0, max_iter=k)
    ref = oracle.jacobi(og, D, tau=0.0, max_iter=k, csc_p=csc_p)
    assert r.iters == k
    assert l1(x, ref.x) <= 1e-13


@pytest.mark.parametrize("variant", ["jacobi", "gs"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_dc", "bf16_dc", "fp16_dc"])
def test_weighted_solves_reach_the_fixed_point(wgraph, variant, precision):
    n, og, csc_p, g, star = wgraph
    x, r = g.solve(variant=variant, precision=precision, threshold=1e-10)
    assert r.status == 0
    bound = BOUND if precision == "fp64" else DC_BOUND
    assert l1(x, star.x) <= bound
    assert abs(float(x.sum()) - 1.0) < 1e-13


def test_weighted_fp32_sweep_and_converged_iterations(wgraph):
    n, og, csc_p, g, star = wgraph
    x, r = g.solve(threshold=1e-10)
    ref = oracle.jacobi(og, D, tau=1e-10, max_iter=1000, csc_p=csc_p)
    assert abs(r.iters - ref.iters) <= 1 and l1(x, ref.x) <= 1e-10
    x32, r32 = g.solve(precision="fp32", threshold=1e-6, max_iter=500)
    assert r32.status == 0 and l1(x32, star.x) < 1e-5


def test_equal_weights_match_the_unweighted_graph():
    n, src, dst = gen.rmat(13, 8, seed=5, dangling_frac=0.1)
    gw = graph(n, src, dst, w=np.full(len(src), 0.37, np.float32))
    gu = graph(n, src, dst)
    for v in ("jacobi", "gs"):
        xw, rw = gw.solve(variant=v, threshold=1e-12)
        xu, ru = gu.solve(variant=v, threshold=1e-12)
        # P = 0.37 / (0.37 outdeg) rounds like 1/outdeg up to one ulp
        assert l1(xw, xu) <= 1e-12
    gw.close()
    gu.close()
