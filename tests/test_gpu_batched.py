"""Batched personalised PageRank (multi right-hand-side FP32 sweep) vs the
oracle's single-teleport Jacobi, column by column."""
import numpy as np
import pytest
import torch

import gen
import oracle
from gpu_util import D, dev, graph, l1

pytestmark = pytest.mark.gpu

TAU = 1e-8
# ||x - x*||_1 <= d/(1-d) tau after the stop, plus the FP32 rounding of the
# sweep map (stored values and sums round at 2^-24 relative; the fixed point
# of the rounded map moves by at most 1/(1-d) times the per-sweep rounding,
# a few 1e-7 in L1 on these graphs): 1e-6 covers both.
FP32_BOUND = D / (1 - D) * TAU + 1e-6


def ppr_ref(og, s):
    tele = np.zeros(og.n)
    tele[s] = 1.0
    star = oracle.fixed_point(og, D, tele=tele, dangling_along_tele=True)
    run = oracle.jacobi(og, D, tau=TAU, max_iter=1000, tele=tele, dangling_along_tele=True)
    return star, run


@pytest.fixture(scope="module")
def s12():
    n, src, dst = gen.rmat(12, 8, seed=3, dangling_frac=0.1)
    og = oracle.build_graph(n, src, dst)
    g = graph(n, src, dst)
    yield n, src, dst, og, g
    g.close()


@pytest.mark.parametrize("B", [1, 40, 128, 300])
def test_batched_fp64_columns_match_single_teleport_solves(s12, B):
    """FP64: every column follows the oracle's single-teleport Jacobi (same
    stop rule), checked on sampled columns across the passes of 128."""
    n, src, dst, og, g = s12
    seeds = gen.seed_vertices(B, n, seed=B)
    X, res = g.solve_batched(dev(seeds), threshold=TAU, precision="fp64")
    assert X.dtype == torch.float64 and X.shape == (n, B)
    Xh = X.cpu().numpy()
    for b in sorted(set(range(B)) & {0, 1, B // 2, B - 1, 37, 127, 128, 255, 256, 299}):
        star, run = ppr_ref(og, int(seeds[b]))
        r = res[b]
        assert r.status == 0, (b, r.iters, r.residual)
        assert abs(r.iters - run.iters) <= 1, (b, r.iters, run.iters)
        assert l1(Xh[:, b], run.x) <= 1e-12
        assert l1(Xh[:, b], star.x) <= D / (1 - D) * TAU * 1.01
        assert abs(Xh[:, b].sum() - 1.0) < 1e-13


@pytest.mark.parametrize("B", [1, 40, 128, 300])
def test_batched_fp32_columns_reach_the_fixed_point(s12, B):
    """FP32: each column ends within the stop bound plus FP32 rounding of the
    fixed point (a column whose change stalls at its rounding floor stops as
    not converged, with the same accuracy)."""
    n, src, dst, og, g = s12
    seeds = gen.seed_vertices(B, n, seed=B)
    X, res = g.solve_batched(dev(seeds), threshold=TAU)
    Xh = X.cpu().numpy().astype(np.float64)
    assert X.dtype == torch.float32 and Xh.shape == (n, B)
    assert sum(r.status == 0 for r in res) >= 0.9 * B
    for b in sorted(set(range(B)) & {0, 1, B // 2, B - 1, 37, 255, 256, 299}):
        star, run = ppr_ref(og, int(seeds[b]))
        r = res[b]
        assert r.status in (0, 4)
        assert r.status == 4 or r.residual <= TAU
        assert l1(Xh[:, b], star.x) <= FP32_BOUND, b
        assert abs(Xh[:, b].sum() - 1.0) < 1e-5
        assert Xh[seeds[b], b] >= (1 - D) * 0.999  # the seed keeps at least 1-d


def test_batched_weighted_and_host_loop(s12):
    n, src, dst, og, _ = s12
    w = gen.edge_weights(len(src), seed=7)
    gw = graph(n, src, dst, w=w)
    _, _, csc_p = oracle.row_normalize(og, w)
    seeds = gen.seed_vertices(33, n, seed=11)
    Xa, ra = gw.solve_batched(dev(seeds), threshold=TAU)
    Xb, rb = gw.solve_batched(dev(seeds), threshold=TAU, use_graph=False)
    assert torch.equal(Xa, Xb)  # same sweeps, deterministic sums
    for b in (0, 17, 32):
        tele = np.zeros(n)
        tele[seeds[b]] = 1.0
        star = oracle.fixed_point(og, D, csc_p=csc_p, tele=tele, dangling_along_tele=True)
        assert ra[b].status in (0, 4)
        assert l1(Xa[:, b].cpu().numpy(), star.x) <= FP32_BOUND
    X64, r64 = gw.solve_batched(dev(seeds), threshold=TAU, precision="fp64")
    for b in (0, 17, 32):
        tele = np.zeros(n)
        tele[seeds[b]] = 1.0
        run = oracle.jacobi(og, D, tau=TAU, max_iter=1000, csc_p=csc_p, tele=tele,
                            dangling_along_tele=True)
        assert r64[b].status == 0 and abs(r64[b].iters - run.iters) <= 1
        assert l1(X64[:, b].cpu().numpy(), run.x) <= 1e-12
    gw.close()


def test_batched_duplicate_seeds_and_max_iter(s12):
    n, src, dst, og, g = s12
    seeds = np.array([5, 5, 9], np.int32)
    X, res = g.solve_batched(dev(seeds), threshold=TAU)
    assert torch.equal(X[:, 0], X[:, 1])
    X, res = g.solve_batched(dev(seeds), threshold=TAU, max_iter=3)
    assert all(r.status == 4 and r.iters == 3 for r in res)
    X, res = g.solve_batched(dev(seeds), threshold=TAU, max_iter=3, precision="fp64")
    assert all(r.status == 4 and r.iters == 3 for r in res)


def test_batched_rejects_bad_seed(s12):
    import paper_2203_09284_gb300 as fp
    n, src, dst, og, g = s12
    with pytest.raises(fp.PageRankError) as e:
        g.solve_batched(dev(np.array([0, n], np.int32)))
    assert e.value.status == fp.PR_ERR_INVALID_ARG
    with pytest.raises(fp.PageRankError) as e:
        g.solve_batched(dev(np.array([0], np.int32)), precision="fp32_dc")
    assert e.value.status == fp.PR_ERR_UNSUPPORTED


def test_batched_full_size_s20_sampled():
    """R-MAT scale 20 with 256 one-hot teleports at the 1e-8 stop (iterates of
    1 GB, beyond L2): sampled FP32 columns against the oracle's single-teleport
    fixed point, sampled FP64 columns against the oracle's Jacobi with the
    same stop."""
    n, src, dst = gen.rmat(20, 16, seed=4)
    og = oracle.build_graph(n, src, dst)
    g = graph(n, src, dst)
    seeds = gen.seed_vertices(256, n, seed=1)
    X, res = g.solve_batched(dev(seeds), threshold=TAU)
    assert sum(r.status == 0 for r in res) >= 0.9 * 256
    X64, r64 = g.solve_batched(dev(seeds), threshold=TAU, precision="fp64")
    assert all(r.status == 0 for r in r64)
    for b in (0, 131, 255):
        tele = np.zeros(n)
        tele[seeds[b]] = 1.0
        star = oracle.fixed_point(og, D, tele=tele, dangling_along_tele=True, max_iter=400)
        assert l1(X[:, b].cpu().numpy(), star.x) <= FP32_BOUND, b
        run = oracle.jacobi(og, D, tau=TAU, max_iter=1000, tele=tele, dangling_along_tele=True)
        assert abs(r64[b].iters - run.iters) <= 1
        assert l1(X64[:, b].cpu().numpy(), run.x) <= 1e-12, b
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_dense_teleport_vectors(s12, precision):
    """Dense teleport vectors V: every column against the oracle's Jacobi with
    that teleport (dangling mass along it); one-hot columns of V give exactly
    the seeds path's result."""
    import paper_2203_09284_gb300 as fp
    n, src, dst, og, g = s12
    B = 6
    rng = np.random.default_rng(7)
    V = np.zeros((n, B))
    V[:, 0] = 1.0 / n                                     # uniform: plain PageRank
    V[:, 1] = rng.random(n)
    V[rng.random(n) < 0.9, 2] = 0.0                       # sparse
    V[:, 2] += (np.arange(n) == 5)
    V[:, 3:] = rng.random((n, B - 3)) ** 4
    V /= V.sum(axis=0)
    dt = np.float64 if precision == "fp64" else np.float32
    X, res = g.solve_batched(V=dev(V.astype(dt)), threshold=TAU, precision=precision)
    Xh = X.cpu().numpy()
    for b in range(B):
        tele = V[:, b].astype(dt).astype(np.float64)
        run = oracle.jacobi(og, D, tau=TAU, max_iter=1000, tele=tele / tele.sum(),
                            dangling_along_tele=True)
        if precision == "fp64":
            assert res[b].status == 0 and abs(res[b].iters - run.iters) <= 1
            assert l1(Xh[:, b], run.x) <= 1e-12, b
        else:
            assert l1(Xh[:, b], run.x) <= FP32_BOUND, b
    seeds = gen.seed_vertices(4, n, seed=2)
    onehot = np.zeros((n, 4), dt)
    onehot[seeds, np.arange(4)] = 1
    Xa, _ = g.solve_batched(dev(seeds), threshold=TAU, precision=precision)
    Xb, _ = g.solve_batched(V=dev(onehot), threshold=TAU, precision=precision)
    assert torch.equal(Xa, Xb)
    bad = onehot.copy()
    bad[0, 0] = -1
    with pytest.raises(fp.PageRankError) as e:
        g.solve_batched(V=dev(bad), precision=precision)
    assert e.value.status == fp.PR_ERR_INVALID_ARG


@pytest.mark.parametrize("precision,B", [("fp32", 300), ("fp64", 140)])
def test_batched_dense_teleport_across_passes(s12, precision, B):
    """Dense V wider than one pass (256 FP32 / 128 FP64 columns): sampled
    columns of every pass against the oracle's Jacobi with that teleport."""
    n, src, dst, og, g = s12
    rng = np.random.default_rng(B)
    dt = np.float64 if precision == "fp64" else np.float32
    V = (rng.random((n, B)) ** 6).astype(dt)
    V /= V.sum(axis=0, dtype=np.float64).astype(dt)
    X, res = g.solve_batched(V=dev(V), threshold=TAU, precision=precision)
    Xh = X.cpu().numpy()
    for b in sorted({0, 1, 127, 128, 129, 255, 256, B - 1} & set(range(B))):
        tele = V[:, b].astype(np.float64)
        run = oracle.jacobi(og, D, tau=TAU, max_iter=1000, tele=tele / tele.sum(),
                            dangling_along_tele=True)
        tol = 1e-12 if precision == "fp64" else FP32_BOUND
        assert l1(Xh[:, b], run.x) <= tol, b
        assert abs(Xh[:, b].sum() - 1) < (1e-13 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batched_split_keeps_every_column_exact(precision):
    """72 of the 128 seeds are dangling vertices, whose columns converge far
    more slowly than the others (about 92 against 16-23 sweeps on this
    graph).  Once the fast ones have stopped, the 128-column pass writes them
    out and hands its 72 running columns to a 64-column pass and a 32-column
    one.  A column's arithmetic does not depend on the pass it is in: every
    column equals its seed solved alone, bit for bit, with the same sweep
    count and residual; one-hot teleport vectors in V (handed over with
    their columns) give the same result; sampled columns match the oracle."""
    n, src, dst = gen.rmat(12, 8, seed=5)          # about 40% of the vertices dangling
    og = oracle.build_graph(n, src, dst)
    g = graph(n, src, dst)
    outdeg = np.bincount(src, minlength=n)
    dangling, live = np.flatnonzero(outdeg == 0), np.flatnonzero(outdeg > 0)
    seeds = np.concatenate([dangling[:72], live[::max(1, len(live) // 56)][:56]]).astype(np.int32)
    seeds = seeds[np.random.default_rng(3).permutation(len(seeds))]
    slow = np.isin(seeds, dangling)
    X, res = g.solve_batched(dev(seeds), threshold=TAU, precision=precision)
    its = np.array([r.iters for r in res])
    assert its[~slow].max() * 2 < its[slow].min()   # two groups: the split happens
    for b in range(len(seeds)):
        Xb, rb = g.solve_batched(dev(seeds[b:b + 1]), threshold=TAU, precision=precision)
        assert torch.equal(X[:, b], Xb[:, 0]), b
        assert res[b].iters == rb[0].iters and res[b].status == rb[0].status, b
        assert res[b].residual == rb[0].residual, b
    dt = np.float64 if precision == "fp64" else np.float32
    onehot = np.zeros((n, len(seeds)), dt)
    onehot[seeds, np.arange(len(seeds))] = 1
    Xv, rv = g.solve_batched(V=dev(onehot), threshold=TAU, precision=precision)
    assert torch.equal(X, Xv)
    assert [r.iters for r in rv] == list(its)
    Xh = X.cpu().numpy()
    for b in range(0, len(seeds), 9):
        tele = np.zeros(n)
        tele[seeds[b]] = 1.0
        run = oracle.jacobi(og, D, tau=TAU, max_iter=1000, tele=tele, dangling_along_tele=True)
        if precision == "fp64":
            assert abs(res[b].iters - run.iters) <= 1 and l1(Xh[:, b], run.x) <= 1e-12, b
        else:
            star = oracle.fixed_point(og, D, tele=tele, dangling_along_tele=True, max_iter=400)
            assert l1(Xh[:, b], star.x) <= FP32_BOUND, b
    g.close()
