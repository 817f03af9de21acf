"""Pins the oracle's iterations (Algorithm 1 / Eq. 2 and Algorithm 2 / Eq. 9)
to closed forms, dense linear solves (numpy and the Perron eigenvector of the
Google matrix), exact rational arithmetic and invariants."""
import os
from fractions import Fraction

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
D = 0.85


def _fixture(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            key, *vals = line.split()
            out[key] = vals
    return out


def _solve(n, src, dst, gs=False, x0=None, tau=1e-15, norm=oracle.NORM_L1, max_iter=3000):
    g = oracle.build_graph(n, src, dst)
    fn = oracle.gauss_seidel if gs else oracle.jacobi
    return g, fn(g, D, tau=tau, max_iter=max_iter, norm=norm, x0=x0)


# --- closed forms ---------------------------------------------------------

@pytest.mark.parametrize("gs", [False, True])
@pytest.mark.parametrize("n", [2, 3, 17, 1000])
def test_cycle_is_uniform(n, gs):
    x0 = gen.random_x0(n, seed=n)
    _, r = _solve(*gen.cycle(n), gs=gs, x0=x0, tau=0.0, max_iter=400)
    # FP64 fixed point of fl((1-d)/n + d x) sits within ulp/(1-d) of 1/n; the
    # final division by the (sequentially summed) total adds <= n eps.
    assert np.max(np.abs(r.x - 1.0 / n)) <= 1e-14 / n


@pytest.mark.parametrize("gs", [False, True])
@pytest.mark.parametrize("leaves", [1, 5, 100])
def test_in_star(leaves, gs):
    n = leaves + 1
    _, r = _solve(*gen.in_star(leaves), gs=gs)
    centre = (1 + (n - 1) * D) / (n + (n - 1) * D)
    leaf = 1 / (n + (n - 1) * D)
    assert abs(r.x[0] - centre) < 1e-13
    assert np.max(np.abs(r.x[1:] - leaf)) < 1e-13


@pytest.mark.parametrize("gs", [False, True])
@pytest.mark.parametrize("leaves", [1, 4, 50])
def test_bidirectional_star(leaves, gs):
    n = leaves + 1
    _, r = _solve(*gen.bi_star(leaves), gs=gs)
    centre = (1 - D + n * D) / (n * (1 + D))
    assert abs(r.x[0] - centre) < 1e-13
    assert np.max(np.abs(r.x[1:] - (1 - centre) / leaves)) < 1e-13


@pytest.mark.parametrize("gs", [False, True])
def test_complete_and_empty_graphs_are_uniform(gs):
    for n, src, dst in [gen.complete(6), (7, np.zeros(0, np.int32), np.zeros(0, np.int32))]:
        _, r = _solve(n, src, dst, gs=gs)
        assert np.max(np.abs(r.x - 1.0 / n)) < 1e-15


@pytest.mark.parametrize("gs", [False, True])
def test_two_vertex_chain(gs):
    _, r = _solve(*gen.chain2(), gs=gs)
    assert abs(r.x[0] - 1 / (2 + D)) < 1e-15
    assert abs(r.x[1] - (1 + D) / (2 + D)) < 1e-15


# --- dense systems (n <= 8) -----------------------------------------------

def _small_graphs():
    cases = []
    for n in range(1, 9):
        for k, p in enumerate([0.2, 0.45, 0.8]):
            cases.append(gen.random_digraph(n, p, seed=100 * n + k, self_loops=(k == 1),
                                            multi=(k == 2)))
    return cases


def _google_perron(n, src, dst, d, tele=None, along=False):
    """Perron vector of the Google matrix G = d M + (1-d) v 1^T, with M built
    column by column from the adjacency (dangling columns = w)."""
    A = np.zeros((n, n))
    for s, t in zip(src, dst):
        A[t, s] += 1.0
    colsum = A.sum(axis=0)
    v = np.full(n, 1.0 / n) if tele is None else np.asarray(tele, float)
    wv = v if along else np.full(n, 1.0 / n)
    M = np.where(colsum > 0, A / np.where(colsum > 0, colsum, 1.0), wv[:, None])
    G = d * M + (1 - d) * np.outer(v, np.ones(n))
    vals, vecs = np.linalg.eig(G)
    k = np.argmin(np.abs(vals - 1.0))
    x = np.real(vecs[:, k])
    return x / x.sum()


@pytest.mark.parametrize("case", range(24))
def test_dense_solve_against_numpy_and_perron(case):
    n, src, dst = _small_graphs()[case]
    A, b = oracle.dense_system(n, src, dst, D)
    x = oracle.dense_solve(A, b)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-14)
    assert np.allclose(x, _google_perron(n, src, dst, D), rtol=0, atol=1e-12)
    assert abs(x.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("gs", [False, True])
@pytest.mark.parametrize("case", range(24))
def test_iterations_reach_dense_solution(case, gs):
    n, src, dst = _small_graphs()[case]
    x_dense = oracle.dense_pagerank(n, src, dst, D)
    g, r = _solve(n, src, dst, gs=gs, tau=1e-15)
    assert r.status == oracle.OK
    assert np.abs(r.x - x_dense).sum() < 1e-13
    assert abs(r.sum_before - 1.0) < 1e-12
    assert (r.x >= (1 - D) / n * (1 - 1e-12)).all()


# --- exact rational arithmetic ---------------------------------------------

def test_gauss_seidel_order_example_of_section_4():
    f = _fixture("gs_order_fig2.txt")
    n = int(f["n"][0])
    d = float(Fraction(f["d"][0]))
    e = np.array([int(v) for v in f["edges"]], np.int32).reshape(-1, 2)
    g = oracle.build_graph(n, e[:, 0], e[:, 1])
    gs = oracle.gauss_seidel(g, d, tau=-1, max_iter=1, normalize=False, renorm=False)
    ja = oracle.jacobi(g, d, tau=-1, max_iter=1, normalize=False)
    for got, key in [(gs.x, "gs_sweep1"), (ja.x, "jacobi_sweep1")]:
        want = np.array([float(Fraction(v)) for v in f[key]])
        assert np.max(np.abs(got - want) / want) <= 2.3e-16


def test_jacobi_trajectory_is_exact_to_rounding():
    """Iterates after k sweeps agree with exact rationals on a small graph."""
    n, src, dst = gen.random_digraph(6, 0.4, seed=11)
    g = oracle.build_graph(n, src, dst)
    d = Fraction(17, 20)
    outdeg = np.bincount(src, minlength=n)
    x = [Fraction(1, n)] * n
    for k in range(1, 9):
        dang = sum(x[u] for u in range(n) if outdeg[u] == 0)
        new = []
        for u in range(n):
            s = sum(x[v] / int(outdeg[v]) for v, t in zip(src, dst) if t == u)
            new.append((1 - d) / n + d * (s + dang / n))
        x = new
        r = oracle.jacobi(g, 0.85, tau=-1, max_iter=k, normalize=False)
        exact = np.array([float(v) for v in x])
        assert np.max(np.abs(r.x - exact) / exact) < 1e-14


def _exact_fused(n, src, dst, d, sweeps, rescale):
    """Eq. 9 in exact rationals: vertices in increasing id order, each in-list
    sum reading the contributions as they stand (already rewritten for
    in-neighbours j < i, old for j >= i), dangling mass D taken at the start of
    the sweep and spread uniformly; with rescale, each sweep ends with x /= sum
    x.  Returns the iterate and each sweep's L1 change (new value against the
    value it replaced, before any rescale)."""
    outdeg = np.bincount(src, minlength=n)
    ins = [[int(v) for v, t in zip(src, dst) if t == u] for u in range(n)]
    x = [Fraction(1, n)] * n
    c = [x[v] / int(outdeg[v]) if outdeg[v] else Fraction(0) for v in range(n)]
    errs = []
    for _ in range(sweeps):
        dang = sum(x[u] for u in range(n) if outdeg[u] == 0)
        err = Fraction(0)
        for u in range(n):
            new = (1 - d) / n + d * (sum(c[v] for v in ins[u]) + dang / n)
            err += abs(new - x[u])
            x[u] = new
            c[u] = new / int(outdeg[u]) if outdeg[u] else Fraction(0)
        errs.append(err)
        if rescale:
            s = sum(x)
            x = [v / s for v in x]
            c = [x[v] / int(outdeg[v]) if outdeg[v] else Fraction(0) for v in range(n)]
    return x, errs


@pytest.mark.parametrize("rescale", [False, True])
@pytest.mark.parametrize("seed", [3, 12])
def test_fused_trajectory_is_exact_to_rounding(seed, rescale):
    """The oracle's sequential fused sweep, with and without the per-sweep
    rescale to sum 1, against exact rationals after 1-4 sweeps on small graphs
    with dangling vertices (where the rescale and the dangling term matter)
    and a self-loop (Eq. 9 reads its own old value)."""
    n, src, dst = gen.random_digraph(7, 0.3, seed=seed, self_loops=True)
    outdeg = np.bincount(src, minlength=n)
    assert (outdeg == 0).any() and (src == dst).any()
    g = oracle.build_graph(n, src, dst)
    for k in range(1, 5):
        x, errs = _exact_fused(n, src, dst, Fraction(17, 20), k, rescale)
        r = oracle.gauss_seidel(g, 0.85, tau=-1, max_iter=k, normalize=False, renorm=rescale)
        exact = np.array([float(v) for v in x])
        assert np.max(np.abs(r.x - exact) / exact) < 1e-14, k
        want = np.array([float(e) for e in errs])
        assert np.allclose(r.history, want, rtol=1e-13, atol=0), k
    # without the rescale the sum drifts (dangling mass read at sweep start,
    # in-neighbours read partly updated values); with it the sum stays 1
    x, _ = _exact_fused(n, src, dst, Fraction(17, 20), 3, rescale)
    if rescale:
        assert sum(x) == 1
    else:
        assert sum(x) != 1


# --- invariants and agreement between variants -----------------------------

@pytest.mark.parametrize("seed", [1, 2])
def test_rmat_jacobi_gs_same_fixed_point(seed):
    n, src, dst = gen.rmat(12, 16, seed=seed)
    g = oracle.build_graph(n, src, dst)
    ja = oracle.jacobi(g, D, tau=1e-13, max_iter=1000)
    gs = oracle.gauss_seidel(g, D, tau=1e-13, max_iter=1000)
    star = oracle.fixed_point(g, D)
    bound = D / (1 - D) * star.err
    assert bound < 1e-14
    assert np.abs(ja.x - star.x).sum() <= D / (1 - D) * 1e-13 + bound
    assert np.abs(gs.x - star.x).sum() <= 1e-11
    assert gs.iters < ja.iters  # fewer sweeps (Sec. 5.3 observation)
    assert abs(ja.sum_before - 1.0) < 1e-12
    assert abs(gs.sum_before - 1.0) < 1e-12


def test_fixed_point_independent_of_start():
    n, src, dst = gen.rmat(10, 8, seed=7)
    g = oracle.build_graph(n, src, dst)
    a = oracle.fixed_point(g, D)
    b = oracle.fixed_point(g, D, x0=gen.random_x0(n, 3))
    assert np.abs(a.x - b.x).sum() < 1e-13


def test_stop_rule_and_history():
    n, src, dst = gen.rmat(10, 8, seed=7)
    g = oracle.build_graph(n, src, dst)
    r = oracle.jacobi(g, D, tau=1e-10, max_iter=500)
    assert r.history[-1] <= 1e-10 < r.history[-2]
    assert len(r.history) == r.iters
    # max_iter reached: not converged, last iterate returned
    r2 = oracle.jacobi(g, D, tau=1e-10, max_iter=5)
    assert r2.status == oracle.NOT_CONVERGED and r2.iters == 5
    # max-norm stop (Eq. 3)
    r3 = oracle.jacobi(g, D, tau=1e-12, norm=oracle.NORM_LINF, max_iter=500)
    assert r3.history[-1] <= 1e-12
    # a tie with the threshold stops (while error > threshold)
    r4 = oracle.jacobi(g, D, tau=r.history[3], max_iter=500)
    assert r4.iters == 4


# --- personalised PageRank --------------------------------------------------

def test_ppr_dense_and_linearity():
    # no dangling vertices: PPR is linear in the teleport vector
    n, src, dst = gen.random_digraph(8, 0.5, seed=21)
    assert (np.bincount(src, minlength=n) > 0).all()
    g = oracle.build_graph(n, src, dst)
    acc = np.zeros(n)
    for s in range(n):
        v = np.zeros(n)
        v[s] = 1.0
        r = oracle.jacobi(g, D, tau=1e-15, max_iter=3000, tele=v, dangling_along_tele=True)
        assert np.abs(r.x - oracle.dense_pagerank(n, src, dst, D, tele=v,
                                                  dangling_along_tele=True)).sum() < 1e-13
        assert np.abs(r.x - _google_perron(n, src, dst, D, tele=v, along=True)).sum() < 1e-12
        acc += r.x
    uni = oracle.jacobi(g, D, tau=1e-15, max_iter=3000)
    assert np.abs(acc / n - uni.x).sum() < 1e-13


def test_ppr_with_dangling_matches_dense():
    n, src, dst = gen.random_digraph(7, 0.3, seed=5)
    g = oracle.build_graph(n, src, dst)
    assert (g.outdeg == 0).any()
    v = np.zeros(n)
    v[2] = 1.0
    for along in (False, True):
        r = oracle.jacobi(g, D, tau=1e-15, max_iter=3000, tele=v, dangling_along_tele=along,
                          normalize=False)
        dense = oracle.dense_pagerank(n, src, dst, D, tele=v, dangling_along_tele=along)
        assert np.abs(r.x - dense).sum() < 1e-13


# --- loop perforation -------------------------------------------------------

def _exact_perforated(n, src, dst, d, eps, period, sweeps):
    """The perforation rule in exact rationals: in a perforated sweep a vertex
    whose change at its last computation was below eps times its value keeps
    that value; every period-th sweep (and the first) is a full Jacobi
    sweep.  Returns the iterates, the per-sweep L1 changes and the skip sets."""
    outdeg = np.bincount(src, minlength=n)
    ins = [[int(v) for v, t in zip(src, dst) if t == u] for u in range(n)]
    x = [Fraction(1, n)] * n
    last = [None] * n  # None: never computed (infinite)
    errs, skips, margins = [], [], []
    for k in range(sweeps):
        full = (period > 0 and k % period == 0) or k == 0
        dang = sum(x[u] for u in range(n) if outdeg[u] == 0)
        c = [x[v] / int(outdeg[v]) if outdeg[v] else Fraction(0) for v in range(n)]
        new, skip, err = list(x), set(), Fraction(0)
        for u in range(n):
            if not full and last[u] is not None:
                margins.append(abs(last[u] - eps * x[u]) / (eps * x[u]))
                if last[u] < eps * x[u]:
                    skip.add(u)
                    continue
            new[u] = (1 - d) / n + d * (sum(c[v] for v in ins[u]) + dang / n)
            last[u] = abs(new[u] - x[u])
            err += last[u]
        x = new
        errs.append(err)
        skips.append(skip)
    return x, errs, skips, margins


def test_perforated_is_jacobi_without_skips():
    n, src, dst = gen.rmat(10, 8, seed=3, dangling_frac=0.2)
    g = oracle.build_graph(n, src, dst)
    ja = oracle.jacobi(g, D, tau=1e-12, max_iter=500)
    for eps, period in ((0.0, 0), (1e-3, 1)):
        r = oracle.perforated(g, D, eps=eps, period=period, tau=1e-12, max_iter=500)
        assert r.iters == ja.iters and np.array_equal(r.x, ja.x)
        assert np.array_equal(r.history, ja.history)
        assert r.gathered == ja.iters * g.m
    # no skips, but only every third sweep may stop: the same sweeps,
    # continued to the next full one
    r = oracle.perforated(g, D, eps=0.0, period=3, tau=1e-12, max_iter=500)
    assert r.iters == ja.iters + (-(ja.iters - 1)) % 3 and (r.iters - 1) % 3 == 0
    assert np.array_equal(r.history[:ja.iters], ja.history)
    assert r.gathered == r.iters * g.m


@pytest.mark.parametrize("period", [0, 3])
def test_perforated_trajectory_is_exact_to_rounding(period):
    """Iterates, per-sweep changes and the number of gathered in-list entries
    against the rule in exact rationals; eps is chosen so that vertices are
    skipped (and no skip decision lies within rounding of the threshold)."""
    n, src, dst = gen.random_digraph(8, 0.3, seed=7)
    g = oracle.build_graph(n, src, dst)
    eps = Fraction(1, 20)
    indeg = np.bincount(dst, minlength=n)
    x, errs, skips, margins = _exact_perforated(n, src, dst, Fraction(17, 20), eps, period, 9)
    assert sum(len(s) for s in skips) >= 5 and min(margins) > 1e-9
    for k in range(1, 10):
        r = oracle.perforated(g, 0.85, eps=float(eps), period=period, tau=-1, max_iter=k,
                              normalize=False)
        xk, ek, sk, _ = _exact_perforated(n, src, dst, Fraction(17, 20), eps, period, k)
        exact = np.array([float(v) for v in xk])
        assert np.max(np.abs(r.x - exact) / exact) < 1e-14, k
        assert np.allclose(r.history, [float(e) for e in ek], rtol=1e-13, atol=0), k
        assert r.gathered == sum(int(indeg.sum()) - int(indeg[list(s)].sum()) for s in sk), k


def test_perforated_full_sweep_stop_certifies_the_bound():
    """With period > 0 the iteration stops only after a full Jacobi sweep, so
    the stop rule's a-posteriori bound d/(1-d) tau holds; with period 0 the
    result is approximate (the skipped vertices' changes are not counted)
    and fewer in-list entries are summed."""
    n, src, dst = gen.rmat(12, 16, seed=2, dangling_frac=0.1)
    g = oracle.build_graph(n, src, dst)
    star = oracle.fixed_point(g, D)
    ja = oracle.jacobi(g, D, tau=1e-10, max_iter=500)
    for eps in (1e-9, 1e-7):
        r = oracle.perforated(g, D, eps=eps, period=4, tau=1e-10, max_iter=2000)
        assert r.status == oracle.OK and (r.iters - 1) % 4 == 0
        assert np.abs(r.x - star.x).sum() <= D / (1 - D) * 1e-10
        a = oracle.perforated(g, D, eps=eps, period=0, tau=1e-10, max_iter=2000)
        assert a.status == oracle.OK and a.gathered < ja.iters * g.m
