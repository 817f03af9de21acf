"""pr_gather_probe (the gather-rate diagnostic the sweep is measured
against) adds up exactly the gathers it is given."""
import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m_cut", [0, 1, 3])
@pytest.mark.parametrize("hot", [0, 1000, 16384])
def test_gather_probe_sums_the_gathers(m_cut, hot):
    import paper_2203_09284_gb300 as fp
    n, src, _ = gen.rmat(16, 16, seed=3)
    m = len(src) - m_cut  # whole 16-byte groups and a ragged tail
    idx = torch.from_numpy(src[:m].copy()).cuda()
    y = torch.from_numpy(gen.edge_weights(n, seed=7)).cuda()  # seeded values in (0, 1]
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    fp.pr_gather_probe(idx, y, sink, hot)
    torch.cuda.synchronize()
    want = y.double().cpu().numpy()[src[:m]].sum()
    # FP32 sums per lane, then per warp and one atomic per warp
    assert abs(float(sink.item()) - want) <= 1e-5 * want


def test_gather_probe_rejects_bad_arguments():
    import paper_2203_09284_gb300 as fp
    y = torch.ones(100, dtype=torch.float32, device="cuda")
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    idx = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(fp.PageRankError):
        fp.pr_gather_probe(idx, y, sink, hot=101)  # more staged entries than y has
    with pytest.raises(fp.PageRankError):
        fp.pr_gather_probe(idx[1:], y, sink)  # not 16-byte aligned
    fp.pr_gather_probe(idx, y, sink)  # the context is still usable
    torch.cuda.synchronize()
    assert float(sink.item()) == 64.0
    # entries outside [0, n) gather y[0] instead of reading out of bounds
    y2 = torch.arange(1, 101, dtype=torch.float32, device="cuda")
    bad = torch.tensor([100, -1, 5000, 7] + [0] * 4, dtype=torch.int32, device="cuda")
    sink.zero_()
    fp.pr_gather_probe(bad, y2, sink)
    torch.cuda.synchronize()
    assert float(sink.item()) == 1 + 1 + 1 + 8 + 4 * 1
