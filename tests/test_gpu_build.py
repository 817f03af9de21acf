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
