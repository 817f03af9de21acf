"""Pins the oracle's graph build (Sec. 3 storage) to numpy's stable sorts,
bincount and the worked storage example of Sec. 3."""
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fixture(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, *vals = line.split()
        out[key] = vals
    return out


def _check_against_numpy(n, src, dst):
    g = oracle.build_graph(n, src, dst)
    m = len(src)
    eid = np.arange(m)
    assert np.array_equal(g.outdeg, np.bincount(src, minlength=n))
    assert np.array_equal(g.indeg, np.bincount(dst, minlength=n))
    csc = np.lexsort((eid, src, dst))  # by dst, then src, then edge id
    csr = np.lexsort((eid, dst, src))  # by src, then dst, then edge id
    assert np.array_equal(g.csc_eid, csc)
    assert np.array_equal(g.row_idx, src[csc])
    assert np.array_equal(g.csr_eid, csr)
    assert np.array_equal(g.col_idx, dst[csr])
    assert np.array_equal(g.col_ptr, np.concatenate([[0], np.cumsum(g.indeg)]))
    assert np.array_equal(g.row_ptr, np.concatenate([[0], np.cumsum(g.outdeg)]))
    with np.errstate(divide="ignore"):
        inv = np.where(g.outdeg > 0, 1.0 / g.outdeg.astype(np.float64), 0.0)
    assert np.array_equal(g.inv_outdeg.view(np.uint64), inv.view(np.uint64))
    return g


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_build_rmat_matches_numpy_sorts(seed):
    n, src, dst = gen.rmat(12, 16, seed=seed)
    _check_against_numpy(n, src, dst)


def test_build_with_duplicates_and_self_loops():
    n, src, dst = gen.rmat(10, 8, seed=5, dedup=False)
    assert (src == dst).any()
    _check_against_numpy(n, src, dst)
    n, src, dst = gen.random_digraph(7, 0.5, seed=3, self_loops=True, multi=True)
    _check_against_numpy(n, src, dst)


def test_build_edge_cases():
    # empty edge list: everything dangling
    g = _check_against_numpy(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert (g.inv_outdeg == 0).all()
    # single vertex with a self-loop
    _check_against_numpy(1, np.array([0], np.int32), np.array([0], np.int32))
    # all edges into one hub, ids up to n-1, unsorted input
    n = 1000
    src = np.arange(n - 1, 0, -1).astype(np.int32)
    _check_against_numpy(n, src, np.zeros(n - 1, np.int32))
    _check_against_numpy(n, np.zeros(n - 1, np.int32), src)


def test_build_rejects_bad_ids():
    with pytest.raises(ValueError):
        oracle.build_graph(4, np.array([0, 4], np.int32), np.array([1, 2], np.int32))
    with pytest.raises(ValueError):
        oracle.build_graph(4, np.array([0, -1], np.int32), np.array([1, 2], np.int32))
    with pytest.raises(ValueError):
        oracle.build_graph(0, np.zeros(0, np.int32), np.zeros(0, np.int32))


def test_storage_example_of_section_3():
    f = _read_fixture("storage_example.txt")
    n = int(f["n"][0])
    e = np.array([int(v) for v in f["edges"]], np.int32).reshape(-1, 2)
    g = oracle.build_graph(n, e[:, 0], e[:, 1])
    u = int(f["inlist_vertex"][0])
    lo, hi = g.col_ptr[u], g.col_ptr[u + 1]
    assert list(g.row_idx[lo:hi]) == [int(v) for v in f["inlist_sources"]]
    assert list(range(lo, hi)) == [int(v) for v in f["inlist_slots"]]
    offs = g.offset_list()
    for slot, val in zip(f["offsetlist_slots"], f["offsetlist_values"]):
        assert offs[int(slot)] == int(val)


@pytest.mark.parametrize("case", ["rmat", "dups", "empty", "hub"])
def test_relabel_matches_numpy(case):
    if case == "rmat":
        n, src, dst = gen.rmat(12, 16, seed=2)
    elif case == "dups":
        n, src, dst = gen.rmat(9, 8, seed=3, dedup=False)
    elif case == "empty":
        n, src, dst = 6, np.zeros(0, np.int32), np.zeros(0, np.int32)
    else:
        n = 300
        src = np.arange(n - 1, 0, -1).astype(np.int32)
        dst = np.zeros(n - 1, np.int32)
    g = oracle.build_graph(n, src, dst)
    n2o, rcol, rrow, reid = oracle.relabel(g)
    want = np.argsort(-g.indeg.astype(np.int64), kind="stable")
    assert np.array_equal(n2o, want)
    o2n = np.empty(n, np.int64)
    o2n[want] = np.arange(n)
    ns, nd = o2n[src], o2n[dst]
    order = np.lexsort((np.arange(len(src)), src, nd))  # new dst, input src, edge id
    assert np.array_equal(reid, order)
    assert np.array_equal(rrow, ns[order])
    assert np.array_equal(rcol, np.concatenate([[0], np.cumsum(np.bincount(nd, minlength=n))]))
    # in-degrees in the new order are non-increasing
    assert (np.diff(np.diff(rcol)) <= 0).all()


def test_bins_are_stable_partition():
    n, src, dst = gen.rmat(12, 16, seed=4)
    g = oracle.build_graph(n, src, dst)
    for t_lo, t_hub in [(4, 256), (16, 1024), (0, 0), (10**6, 10**7)]:
        low, mid, hub = oracle.bins(g, t_lo, t_hub)
        ids = np.arange(n)
        assert np.array_equal(low, ids[g.indeg <= t_lo])
        assert np.array_equal(mid, ids[(g.indeg > t_lo) & (g.indeg <= t_hub)])
        assert np.array_equal(hub, ids[g.indeg > t_hub])
