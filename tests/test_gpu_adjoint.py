"""pr_backward (adjoint over the out-lists, edge-weight and damping
gradients) vs the oracle's adjoint and gradients, and vs cancellation-free
central differences of the oracle's forward solve."""
import numpy as np
import pytest
import torch

import gen
import oracle
from gpu_util import D, dev, graph

pytestmark = pytest.mark.gpu


def _loss_grad(n, seed, count):
    t, c = gen.loss_targets(min(count, n), n, seed)
    gx = np.zeros(n)
    gx[t] = c
    return gx


def _oracle(og, w, gx, weighted):
    if weighted:
        s, csr_p, csc_p = oracle.row_normalize(og, w)
    else:
        csr_p = csc_p = None
    x = oracle.fixed_point(og, D, csc_p=csc_p).x
    lam, _, _ = oracle.adjoint(og, gx, D, csr_p=csr_p)
    gw, gd = oracle.gradients(og, x, lam, D, w=w if weighted else None)
    return x, csc_p, gw, gd


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("use_graph", [True, False])
def test_backward_matches_oracle_fp64(weighted, use_graph):
    n, src, dst = gen.rmat(12, 8, seed=21, dangling_frac=0.05)
    w = gen.edge_weights(len(src), seed=3) if weighted else None
    og = oracle.build_graph(n, src, dst)
    gx = _loss_grad(n, 5, 200)
    x, csc_p, gw_ref, gd_ref = _oracle(og, w, gx, weighted)
    g = graph(n, src, dst, w=w)
    xg, r = g.solve(threshold=1e-14, max_iter=2000)
    gw, gd, rb = g.backward(xg, dev(gx), threshold=1e-15, max_iter=5000, use_graph=use_graph)
    assert rb.status in (0, 4)
    gw = gw.cpu().numpy()
    scale = np.abs(gw_ref).max()
    # both sides solve the same systems to round-off; the adjoint's own
    # stop leaves ||lambda - lambda*||_1 <= d/(1-d) * 1e-15 * ||.||
    assert np.abs(gw - gw_ref).max() <= 1e-9 * scale
    assert abs(float(gd) - gd_ref) <= 1e-9 * max(abs(gd_ref), 1e-12)
    g.close()


def test_backward_fp32_and_finite_differences():
    """R-MAT scale 14, raw weights uniform in (0, 1]: FP32 adjoint within
    relative 1e-5 of the FP64 one; FP64 gradients within relative 1e-6 of
    central differences (h = 1e-6) of the oracle on sampled edges and d."""
    n, src, dst = gen.rmat(14, 16, seed=8)
    w = gen.edge_weights(len(src), seed=9)
    og = oracle.build_graph(n, src, dst)
    gx = _loss_grad(n, 11, 1000)
    g = graph(n, src, dst, w=w)
    xg, _ = g.solve(threshold=1e-14, max_iter=2000)
    gw64, gd64, _ = g.backward(xg, dev(gx), threshold=1e-15, max_iter=5000)
    gw32, gd32, r32 = g.backward(xg, dev(gx), precision="fp32", threshold=1e-9, max_iter=2000)
    a, b = gw64.cpu().numpy(), gw32.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()
    assert abs(float(gd32) - float(gd64)) <= 1e-5 * abs(float(gd64))
    x = xg.cpu().numpy()
    _, _, csc_p = oracle.row_normalize(og, w)
    for e in gen.fd_edges(20, len(src), seed=4):
        fd = oracle.fd_weight(og, w, x, gx, int(e), h=1e-6, d=D, csc_p=csc_p)
        assert abs(a[e] - fd) <= 1e-6 * np.abs(a).max() + 1e-6 * abs(fd), (e, a[e], fd)
    fdd = oracle.fd_damping(og, x, gx, h=1e-6, d=D, csc_p=csc_p)
    assert abs(float(gd64) - fdd) <= 1e-6 * abs(fdd)
    g.close()


def test_pagerank_fn_autograd():
    import paper_2203_09284_gb300 as fp
    n, src, dst = gen.rmat(11, 8, seed=31)
    w = torch.from_numpy(gen.edge_weights(len(src), seed=1)).cuda().requires_grad_(True)
    d = torch.tensor(D, dtype=torch.float64, requires_grad=True)
    t, c = gen.loss_targets(100, n, 2)
    x = fp.PageRankFn.apply(w, d, dev(src), dev(dst), n, {"threshold": 1e-14, "max_iter": 2000})
    loss = (x[dev(t.astype(np.int64))] * dev(c)).sum()
    loss.backward()
    og = oracle.build_graph(n, src, dst)
    gx = np.zeros(n)
    gx[t] = c
    _, _, gw_ref, gd_ref = _oracle(og, w.detach().cpu().numpy(), gx, True)
    assert np.abs(w.grad.double().cpu().numpy() - gw_ref).max() <= 1e-6 * np.abs(gw_ref).max()
    assert abs(float(d.grad) - gd_ref) <= 1e-8 * abs(gd_ref)


def test_backward_full_size_s18():
    """R-MAT scale 18, raw weights uniform in (0, 1], 1,000 loss targets with
    coefficients U(-1, 1) (the differentiable workload):
      - the FP64 adjoint's edge-weight gradient against the oracle's adjoint
        and gradients, edge by edge, to relative 1e-6 (floor 1e-12 of the
        largest), and dL/dd likewise;
      - the FP32 adjoint against the same, to 1e-5 of the largest gradient
        (and in relative L2);
      - the FP64 gradient against cancellation-free FP64 central differences
        (h = 1e-6) of the oracle's fixed point on 100 sampled edges and d,
        each to relative 1e-6 plus the solves' own error bound, and to
        relative 1e-6 in L2 over the 100 edges.
    The central differences (two oracle solves each) run in spawned host
    processes while the GPU works."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os

    import oracle_pool
    n, src, dst = gen.rmat(18, 16, seed=18)
    w = gen.edge_weights(len(src), seed=18)
    og = oracle.build_graph(n, src, dst)
    gx = _loss_grad(n, 18, 1000)
    s_, csr_p, csc_p = oracle.row_normalize(og, w)
    xstar = oracle.fixed_point(og, D, csc_p=csc_p).x
    lam, _, _ = oracle.adjoint(og, gx, D, csr_p=csr_p)
    gw_ref, gd_ref = oracle.gradients(og, xstar, lam, D, w=w)
    edges = [int(e) for e in gen.fd_edges(100, len(src), seed=18)]
    workers = max(1, min(16, os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"),
                                initializer=oracle_pool.init_weighted,
                                initargs=(18, 16, 18, 18, xstar, gx, D)) as pool:
        fut_e = [pool.submit(oracle_pool.fd_edge, e) for e in edges]
        fut_d = pool.submit(oracle_pool.fd_damping)
        g = graph(n, src, dst, w=w)
        xg, _ = g.solve(threshold=1e-14, max_iter=2000)
        gw64, gd64, r64 = g.backward(xg, dev(gx), threshold=1e-15, max_iter=5000)
        gw32, gd32, r32 = g.backward(xg, dev(gx), precision="fp32", threshold=1e-9,
                                     max_iter=2000)
        g.close()
        a, b = gw64.cpu().numpy(), gw32.cpu().numpy()
        scale = np.abs(gw_ref).max()
        bad = np.abs(a - gw_ref) > 1e-6 * np.abs(gw_ref) + 1e-12 * scale
        assert not bad.any(), (int(bad.sum()), np.abs(a - gw_ref)[bad][:5], gw_ref[bad][:5])
        assert abs(float(gd64) - gd_ref) <= 1e-6 * abs(gd_ref)
        assert np.abs(b - gw_ref).max() <= 1e-5 * scale
        assert np.linalg.norm(b - gw_ref) <= 1e-5 * np.linalg.norm(gw_ref)
        assert abs(float(gd32) - gd_ref) <= 1e-5 * abs(gd_ref)
        fd = np.array([f.result()[0] for f in fut_e])
        noise = np.array([f.result()[1] for f in fut_e])
        fdd, noise_d = fut_d.result()
    ae = a[edges]
    bad = np.abs(ae - fd) > 1e-6 * np.abs(fd) + noise + 1e-12 * np.abs(fd).max()
    assert not bad.any(), list(zip(np.array(edges)[bad], ae[bad], fd[bad], noise[bad]))
    assert np.linalg.norm(ae - fd) <= 1e-6 * np.linalg.norm(fd)
    assert abs(float(gd64) - fdd) <= 1e-6 * abs(fdd) + noise_d
