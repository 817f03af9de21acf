"""pr_scan_exclusive_noalloc (fixed device scratch, no allocation) against
the offsets the graph build computes with allocated scratch (pr_graph_create
+ pr_graph_export), over two calls in a row.  Collected last so it also runs
after every other test has used the device."""
import numpy as np
import pytest
import torch

import gen
from gpu_util import dev, graph

pytestmark = pytest.mark.gpu

LIMIT = 65536 * 2048


def test_noalloc_scan_matches_build_offsets_twice():
    import paper_2203_09284_gb300 as fp
    n, src, dst = gen.rmat(16, 16, seed=9)
    g = graph(n, src, dst)
    ex = g.export()
    for _ in range(2):
        for key, ptr in (("indeg", "col_ptr"), ("outdeg", None)):
            out = torch.full((n + 1,), -7, dtype=torch.int32, device="cuda")
            fp.pr_scan_exclusive_noalloc(ex[key], out)
            if ptr:
                assert torch.equal(out, ex[ptr])
            else:
                ref = np.concatenate([[0], np.cumsum(ex[key].cpu().numpy())])
                assert np.array_equal(out.cpu().numpy(), ref)
    g.close()


def test_noalloc_scan_sizes_and_limit():
    import paper_2203_09284_gb300 as fp
    rng = np.random.default_rng(3)
    for count in (0, 1, 2047, 2048, 2049, 5 * 2048 + 17, 1 << 22):
        a = rng.integers(0, 100, size=count, dtype=np.int32)
        for _ in range(2):
            out = torch.full((count + 1,), -1, dtype=torch.int32, device="cuda")
            inp = dev(a) if count else torch.empty(0, dtype=torch.int32, device="cuda")
            fp.pr_scan_exclusive_noalloc(inp, out)
            ref = np.concatenate([[0], np.cumsum(a, dtype=np.int64)]).astype(np.int32)
            assert np.array_equal(out.cpu().numpy(), ref), count
    # over the limit: rejected on the host, before any device work
    small = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(fp.PageRankError) as e:
        fp.pr_scan_exclusive_noalloc(small, small, count=LIMIT + 1)
    assert e.value.status == fp.PR_ERR_INVALID_ARG
    with pytest.raises(fp.PageRankError):
        fp.pr_scan_exclusive_noalloc(small, small, count=-1)
