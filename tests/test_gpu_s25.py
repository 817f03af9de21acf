"""R-MAT scale 25 (33.5M vertices, ~537M edges), the crawl-sized mixed
precision workload: BF16- and FP16-stored corrections with FP32 sums and FP64
residuals reach the FP64 stop rule.  Checked on sampled vertices with the
definition of the sweep (each sampled F(x)_u computed directly from the edge
list) and by properties that hold at any size."""
import numpy as np
import pytest
import torch

import gen
from gpu_util import D, dev, graph, l1

pytestmark = pytest.mark.gpu


def sampled_residual(n, src, dst, outdeg, x, sample):
    """sum over sampled u of |F(x)_u - x_u|, F(x)_u = (1-d)/n +
    d (sum_{v -> u} x_v / outdeg(v) + D / n), D the dangling mass of x."""
    Dm = x[outdeg == 0].sum()
    pos = np.full(n, -1, np.int64)
    pos[sample] = np.arange(len(sample))
    sel = pos[dst] >= 0
    s, t = src[sel], pos[dst[sel]]
    acc = np.bincount(t, weights=x[s] / outdeg[s], minlength=len(sample))
    fx = (1 - D) / n + D * (acc + Dm / n)
    return np.abs(fx - x[sample])


def test_rmat25_mixed_precision_reaches_fp64_stop():
    n, src, dst = gen.rmat(25, 16, seed=1)
    g = graph(n, src, dst)
    ex = g.export()
    indeg = np.bincount(dst, minlength=n)
    outdeg = np.bincount(src, minlength=n)
    assert np.array_equal(ex["indeg"].cpu().numpy(), indeg)   # a1, bit-exact
    assert np.array_equal(ex["outdeg"].cpu().numpy(), outdeg)
    cp = ex["col_ptr"].cpu().numpy()
    assert cp[0] == 0 and np.array_equal(np.diff(cp), indeg)  # a2
    del ex
    sample = np.unique(gen.seed_vertices(4096, n, seed=25))
    xs = {}
    for v, prec in (("jacobi", "fp64"), ("jacobi", "bf16_dc"), ("gs", "fp16_dc"),
                    ("gs", "bf16_dc")):
        x, r = g.solve(variant=v, precision=prec, threshold=1e-10)
        assert r.status == 0, (v, prec)
        xh = x.cpu().numpy()
        assert abs(xh.sum() - 1) < 1e-12 and xh.min() >= (1 - D) / n * (1 - 1e-9)
        res = sampled_residual(n, src, dst, outdeg, xh, sample)
        # the whole-graph L1 residual is <= 1e-10 after the stop (the DC stop
        # value is that residual; Jacobi's is d times its last change)
        assert res.sum() <= 1e-10, (v, prec, res.sum())
        xs[(v, prec)] = xh
    ref = xs[("jacobi", "fp64")]
    for k, xh in xs.items():
        # both within ||x - x*||_1 <= 1e-10 / (1 - d) of the fixed point
        assert l1(xh, ref) <= 2e-10 / (1 - D), k
    g.close()
