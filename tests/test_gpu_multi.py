"""Many graphs solved together (one launch per sweep over all graphs' items)
vs each graph's own solve and the oracle."""
import numpy as np
import pytest
import torch

import gen
import oracle
from gpu_util import BOUND, D, graph, l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def family():
    shapes = gen.multi_graph_shapes(7, seed=2, scale_lo=8, scale_hi=13)
    gs, ogs = [], []
    for i, (scale, ef) in enumerate(shapes):
        n, src, dst = gen.rmat(scale, ef, seed=100 + i, dangling_frac=0.05 * (i % 3))
        w = gen.edge_weights(len(src), seed=i) if i == 3 else None
        gs.append(graph(n, src, dst, w=w))
        og = oracle.build_graph(n, src, dst)
        csc_p = oracle.row_normalize(og, w)[2] if w is not None else None
        ogs.append((og, csc_p))
    yield gs, ogs
    for g in gs:
        g.close()


def test_multi_matches_single_solves_and_oracle(family):
    import paper_2203_09284_gb300 as fp
    gs, ogs = family
    xs, res = fp.solve_multi(gs, threshold=1e-10)
    for g, (og, csc_p), x, r in zip(gs, ogs, xs, res):
        assert r.status == 0
        xsingle, rs = g.solve(threshold=1e-10)
        # same items and per-vertex arithmetic; the sweep sums are grouped
        # differently (per item instead of per block) before their exact
        # fixed-point accumulation, which moves them by a few ulp
        assert abs(r.iters - rs.iters) <= 1
        assert l1(x, xsingle) <= 1e-12
        star = oracle.fixed_point(og, D, csc_p=csc_p)
        assert l1(x, star.x) <= BOUND
        ref = oracle.jacobi(og, D, tau=1e-10, max_iter=1000, csc_p=csc_p)
        assert abs(r.iters - ref.iters) <= 1


def test_multi_fixed_sweeps_trajectory(family):
    import paper_2203_09284_gb300 as fp
    gs, ogs = family
    xs, res = fp.solve_multi(gs, threshold=0.0, max_iter=7)
    for (og, csc_p), x, r in zip(ogs, xs, res):
        assert r.status == 4 and r.iters == 7
        ref = oracle.jacobi(og, D, tau=0.0, max_iter=7, csc_p=csc_p)
        assert l1(x, ref.x) <= 1e-13


def test_multi_host_loop_fp32_and_errors(family):
    import paper_2203_09284_gb300 as fp
    gs, ogs = family
    xa, ra = fp.solve_multi(gs, threshold=1e-10)
    xb, rb = fp.solve_multi(gs, threshold=1e-10, use_graph=False)
    for a, b in zip(xa, xb):
        assert torch.equal(a, b)
    xf, rf = fp.solve_multi(gs, precision="fp32", threshold=1e-6, max_iter=300)
    for (og, csc_p), x, r in zip(ogs, xf, rf):
        assert r.status == 0
        assert l1(x, oracle.fixed_point(og, D, csc_p=csc_p).x) < 1e-5
    with pytest.raises(fp.PageRankError):
        fp.solve_multi([gs[0], gs[0]])
    with pytest.raises(fp.PageRankError):
        fp.solve_multi(gs[:2], precision="fp32_dc")
    with pytest.raises(fp.PageRankError):
        fp.solve_multi(gs[:2], perforate_eps=1e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_multi_fused_sweep(family, precision):
    """The fused sweep (Algorithm 2, asynchronous, rescaled) on every graph
    in one launch per sweep: each result within the stop rule's bound of its
    graph's fixed point, in no more sweeps than Jacobi; with no_rescale the
    literal Algorithm 2 reaches the same fixed points."""
    import paper_2203_09284_gb300 as fp
    gs, ogs = family
    tau = 1e-10 if precision == "fp64" else 1e-6
    xj, rj = fp.solve_multi(gs, threshold=tau, precision=precision)
    xg, rg = fp.solve_multi(gs, threshold=tau, precision=precision, variant="gs")
    xl, rl = fp.solve_multi(gs, threshold=tau, precision=precision, variant="gs",
                            no_rescale=True, max_iter=3000)
    for (og, csc_p), x, r, a, b, y, c in zip(ogs, xg, rg, xj, rj, xl, rl):
        assert r.status == 0 and c.status == 0
        star = oracle.fixed_point(og, D, csc_p=csc_p).x
        bound = BOUND if precision == "fp64" else 1e-5
        assert l1(x, star) <= bound
        assert l1(y, star) <= (1e-9 if precision == "fp64" else 1e-5)
        assert r.iters <= b.iters + 1


def test_multi_64_uneven_graphs():
    """64 R-MAT graphs of scale 10 to 18 and edge factor 8 to 32 in one
    solve; sampled graphs against the oracle's fixed point."""
    import paper_2203_09284_gb300 as fp
    shapes = gen.multi_graph_shapes(64, seed=1)
    data, gs = [], []
    for i, (scale, ef) in enumerate(shapes):
        n, src, dst = gen.rmat(scale, ef, seed=1000 + i)
        data.append((n, src, dst))
        gs.append(graph(n, src, dst))
    xs, res = fp.solve_multi(gs, threshold=1e-10)
    assert all(r.status == 0 for r in res)
    for i in (0, 17, 40, 63):
        n, src, dst = data[i]
        og = oracle.build_graph(n, src, dst)
        assert l1(xs[i], oracle.fixed_point(og, D).x) <= BOUND
    for g in gs:
        g.close()
