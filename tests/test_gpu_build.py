"""Device graph build vs the oracle: degrees, offsets, in-lists, out-lists,
inverse out-degrees and bins must match bit for bit."""
import numpy as np
import pytest
import torch

import gen
import oracle
from gpu_util import graph

pytestmark = pytest.mark.gpu


def check_build(n, src, dst, t_lo=32, t_hub=4096):
    g = graph(n, src, dst)
    ex = g.export(csr=True)
    o = oracle.build_graph(n, src, dst)
    c = lambda k: ex[k].cpu().numpy()
    assert np.array_equal(c("outdeg"), o.outdeg)
    assert np.array_equal(c("indeg"), o.indeg)
    assert np.array_equal(c("col_ptr"), o.col_ptr)
    assert np.array_equal(c("row_idx"), o.row_idx)
    assert np.array_equal(c("csc_eid"), o.csc_eid)
    assert np.array_equal(c("row_ptr"), o.row_ptr)
    assert np.array_equal(c("col_idx"), o.col_idx)
    assert np.array_equal(c("csr_eid"), o.csr_eid)
    assert np.array_equal(c("inv_outdeg").view(np.uint64), o.inv_outdeg.view(np.uint64))
    # degree-ordered numbering and its in-lists
    n2o, rcol, rrow, _ = oracle.relabel(o)
    assert np.array_equal(c("new_to_old"), n2o)
    assert np.array_equal(c("rcol_ptr"), rcol)
    assert np.array_equal(c("rrow_idx"), rrow)
    low, mid, hub = oracle.bins(o, t_lo, t_hub)
    info = g.info()
    assert info["n_dangling"] == int((o.outdeg == 0).sum())
    assert info["bins"] == [len(low), len(mid), len(hub)]
    # bin membership: the classes are contiguous ranges of the degree-ordered
    # ids (hubs first, then mid, then low), so each bin's input ids, sorted,
    # are the oracle's bin list
    nh, nm = len(hub), len(mid)
    n2o_g = c("new_to_old")
    assert np.array_equal(np.sort(n2o_g[:nh]), hub)
    assert np.array_equal(np.sort(n2o_g[nh:nh + nm]), mid)
    assert np.array_equal(np.sort(n2o_g[nh + nm:]), low)
    g.close()


@pytest.mark.parametrize("scale,ef,seed", [(10, 16, 1), (16, 16, 1), (17, 5, 2), (18, 16, 3)])
def test_build_rmat(scale, ef, seed):
    check_build(*gen.rmat(scale, ef, seed=seed))


def test_build_duplicates_self_loops_unsorted():
    check_build(*gen.rmat(13, 16, seed=9, dedup=False))
    check_build(*gen.random_digraph(8, 0.6, seed=4, self_loops=True, multi=True))


def test_build_edge_cases():
    check_build(1, np.zeros(0, np.int32), np.zeros(0, np.int32))
    check_build(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    check_build(1, np.array([0, 0], np.int32), np.array([0, 0], np.int32))
    n = 70000  # one hub with every edge: several hub segments, ids up to n-1
    src = np.arange(n - 1, 0, -1).astype(np.int32)
    check_build(n, src, np.zeros(n - 1, np.int32))
    check_build(n, np.zeros(n - 1, np.int32), src)
    check_build(*gen.in_star(5000))


def test_build_rejects_bad_ids():
    import paper_2203_09284_gb300 as fp
    for s, d in (([0, 5], [1, 2]), ([0, 1], [-1, 2])):
        with pytest.raises(fp.PageRankError) as e:
            graph(5, np.array(s, np.int32), np.array(d, np.int32))
        assert e.value.status == fp.PR_ERR_INVALID_ARG
    with pytest.raises(fp.PageRankError):
        graph(4, np.array([0], np.int32), np.array([1], np.int32),
              w=np.array([-1.0], np.float32))
    # the context is still usable afterwards
    check_build(*gen.cycle(10))


def test_build_full_size_rmat22():
    """R-MAT scale 22 (configuration of the web-like workload): bit-exact."""
    check_build(*gen.rmat(22, 16, seed=1, dangling_frac=0.10))


# The edge sort works on tiles of 4096 pairs: full tiles arrive by bulk
# copy, a last partial one by plain loads, and 2 resident blocks per SM take
# tiles round-robin.  Edge counts on and around those boundaries, and more
# tiles than resident blocks.
@pytest.mark.parametrize("m", [1, 4095, 4096, 4097, 8192, 8193, 4096 * 700 + 3])
def test_build_sort_tile_boundaries(m):
    n, src, dst = gen.rmat(18, 16, seed=11)
    assert len(src) >= m
    check_build(n, src[:m], dst[:m])


def test_build_sort_one_hot_digit():
    # every key's low source and destination digits equal (one bucket per
    # tile in those passes), ragged last tile
    n, src, dst = gen.rmat(16, 16, seed=12)
    m = 4096 * 5 + 11
    check_build(n, (src[:m] % 256) * 256, (dst[:m] % 256) * 256)


def test_build_from_pinned_host_arrays():
    """Edge arrays in page-locked host memory are read by the build over the
    host link: the same products as from device arrays (weighted too);
    pageable host arrays are refused before any kernel reads them."""
    import ctypes
    import paper_2203_09284_gb300 as fp
    n, src, dst = gen.rmat(15, 16, seed=5)
    w = gen.edge_weights(len(src), seed=5)
    for weights in (None, w):
        g_dev = graph(n, src, dst, weights, build_csr=True)
        pin = lambda a: torch.from_numpy(a).pin_memory()
        g_pin = fp.Graph(n, pin(src), pin(dst), None if weights is None else pin(weights),
                         build_csr=True)
        a, b = g_dev.export(csr=True), g_pin.export(csr=True)
        assert a.keys() == b.keys()
        for k in a:
            assert torch.equal(a[k], b[k]), k
        x1, r1 = g_dev.solve(threshold=1e-10)
        x2, r2 = g_pin.solve(threshold=1e-10)
        assert r1.iters == r2.iters and torch.equal(x1, x2)
        g_dev.close()
        g_pin.close()
    with pytest.raises(ValueError):
        fp.Graph(n, torch.from_numpy(src), torch.from_numpy(dst))
    out = ctypes.c_void_p()
    st = fp.lib().pr_graph_create(int(n), int(len(src)), ctypes.c_void_p(src.ctypes.data),
                                  ctypes.c_void_p(dst.ctypes.data), None, 0, None,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                  ctypes.byref(out))
    assert st == fp.PR_ERR_INVALID_ARG and not out.value



def test_build_dedup_keeps_first_occurrences():
    """PR_DEDUP: the graph of the first occurrence of every (src, dst) pair,
    bit for bit the oracle's build of that list, with csc_eid giving the kept
    edges' input positions; its solves equal those of the pre-deduplicated
    list, and pr_backward gives the dropped repeats a zero gradient."""
    import paper_2203_09284_gb300 as fp
    for n, src, dst in (gen.rmat(13, 16, seed=9, dedup=False),
                        gen.random_digraph(8, 0.6, seed=4, self_loops=True, multi=True)):
        key = src.astype(np.int64) * n + dst
        _, first = np.unique(key, return_index=True)
        keep = np.sort(first)  # input positions of first occurrences, in input order
        assert len(keep) < len(src)
        g = graph(n, src, dst, dedup=True)
        assert g.info()["m"] == len(keep)
        ex = g.export(csr=True)
        o = oracle.build_graph(n, src[keep], dst[keep])
        c = lambda k: ex[k].cpu().numpy()
        for k in ("outdeg", "indeg", "col_ptr", "row_idx", "row_ptr", "col_idx"):
            assert np.array_equal(c(k), getattr(o, k)), k
        assert np.array_equal(c("csc_eid"), keep[o.csc_eid])
        assert np.array_equal(c("csr_eid"), keep[o.csr_eid])
        assert np.array_equal(c("inv_outdeg").view(np.uint64), o.inv_outdeg.view(np.uint64))
        n2o, rcol, rrow, _ = oracle.relabel(o)
        assert np.array_equal(c("new_to_old"), n2o)
        assert np.array_equal(c("rrow_idx"), rrow)
        g2 = graph(n, src[keep], dst[keep])
        x1, _ = g.solve(threshold=1e-12)
        x2, _ = g2.solve(threshold=1e-12)
        assert torch.equal(x1, x2)
        gx = torch.zeros(n, dtype=torch.float64, device="cuda")
        gx[0] = 1.0
        gw, gd, _ = g.backward(x1, gx, threshold=1e-13)
        gw2, gd2, _ = g2.backward(x2, gx, threshold=1e-13)
        gw = gw.cpu().numpy()
        assert len(gw) == len(src)
        drop = np.setdiff1d(np.arange(len(src)), keep)
        assert (gw[drop] == 0).all()
        assert np.array_equal(gw[keep], gw2.cpu().numpy())
        g.close()
        g2.close()
    with pytest.raises(fp.PageRankError):
        fp.pr_graph_create(4, torch.zeros(1, dtype=torch.int32, device="cuda"),
                           torch.zeros(1, dtype=torch.int32, device="cuda"), flags=4)


def test_build_dedup_weighted():
    """PR_DEDUP with edge weights: the kept edges' weights (first
    occurrences) define P; the solve equals the weighted solve of the
    deduplicated list, and the oracle's weighted fixed point."""
    n, src, dst = gen.rmat(12, 16, seed=4, dedup=False)
    w = gen.edge_weights(len(src), seed=5)
    key = src.astype(np.int64) * n + dst
    _, first = np.unique(key, return_index=True)
    keep = np.sort(first)
    assert len(keep) < len(src)
    g = graph(n, src, dst, w=w, dedup=True)
    g2 = graph(n, src[keep], dst[keep], w=w[keep])
    x1, r1 = g.solve(threshold=1e-13)
    x2, r2 = g2.solve(threshold=1e-13)
    assert torch.equal(x1, x2)
    og = oracle.build_graph(n, src[keep], dst[keep])
    _, _, csc_p = oracle.row_normalize(og, w[keep])
    star = oracle.fixed_point(og, 0.85, csc_p=csc_p)
    assert float(np.abs(x1.cpu().numpy() - star.x).sum()) <= 0.85 / 0.15 * 1e-13 * 1.01
    g.close()
    g2.close()


def test_build_without_allocator_hooks_uses_the_library_pool():
    """A graph created with no allocator hooks takes its memory from the
    library's own pool; built and solved twice in a row (the second build
    reuses the memory the first one freed), it matches the graph built
    through torch's caching allocator exactly."""
    import paper_2203_09284_gb300 as fp
    n, src, dst = gen.rmat(12, 8, seed=9, dangling_frac=0.1)
    ref = graph(n, src, dst)
    xr, rr = ref.solve(threshold=1e-10)
    ea = ref.export()
    for _ in range(2):
        g = graph(n, src, dst, use_torch_allocator=False)
        eb = g.export()
        for k in ea:
            assert torch.equal(ea[k], eb[k]), k
        x, r = g.solve(threshold=1e-10)
        assert r.iters == rr.iters and torch.equal(x, xr)
        xg, rg = g.solve(variant="gs", precision="fp32_dc", threshold=1e-10)
        assert rg.status == 0
        g.close()
    ref.close()
