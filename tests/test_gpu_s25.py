"""R-MAT scale 25 (33.5M vertices, ~537M edges), the crawl-sized mixed
precision workload: FP64 and the BF16-, FP16- and FP32-stored corrections with
FP32 sums and FP64 residuals reach the FP64 stop rule.  Checked over the whole
graph with the definition of the sweep: F(x)_u computed on the host from the
edge list for every vertex, in FP64, and the L1 residual ||F(x) - x||_1,
which bounds the distance to the fixed point: ||x - x*||_1 <= ||F(x) - x||_1 /
(1 - d)."""
import numpy as np
import pytest

import gen
from gpu_util import D, graph, l1

pytestmark = pytest.mark.gpu


def full_residual(n, src, dst, outdeg, x, chunk=1 << 26):
    """||F(x) - x||_1 with F(x)_u = (1-d)/n + d (sum_{v -> u} x_v / outdeg(v)
    + D / n), D the dangling mass of x; the in-edge sums are accumulated in
    FP64 over chunks of the edge list."""
    Dm = x[outdeg == 0].sum()
    c = np.zeros(n)
    nz = outdeg > 0
    c[nz] = x[nz] / outdeg[nz]
    acc = np.zeros(n)
    for a in range(0, len(src), chunk):
        acc += np.bincount(dst[a:a + chunk], weights=c[src[a:a + chunk]], minlength=n)
    fx = (1 - D) / n + D * (acc + Dm / n)
    return float(np.abs(fx - x).sum())


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
    del ex, cp
    xs = {}
    for v, prec, limit in (("jacobi", "fp64", 0.8501e-10), ("jacobi", "fp32_dc", 1.0001e-10),
                           ("jacobi", "bf16_dc", 1.0001e-10), ("jacobi", "fp16_dc", 1.0001e-10),
                           ("gs", "fp16_dc", 1.0001e-10), ("gs", "bf16_dc", 1.0001e-10)):
        x, r = g.solve(variant=v, precision=prec, threshold=1e-10)
        assert r.status == 0, (v, prec)
        xh = x.cpu().numpy()
        assert abs(xh.sum() - 1) < 1e-12 and xh.min() >= (1 - D) / n * (1 - 1e-9)
        # the DC stop value is this residual; Jacobi's is d times its last change
        res = full_residual(n, src, dst, outdeg, xh)
        assert res <= limit, (v, prec, res)
        xs[(v, prec)] = (xh, res)
    # any two results lie within the sum of their certified distances to x*
    items = list(xs.items())
    for i in range(len(items)):
        for j in range(i + 1, len(items)):
            (ka, (xa, ra)), (kb, (xb, rb)) = items[i], items[j]
            assert l1(xa, xb) <= (ra + rb) / (1 - D) * 1.0001, (ka, kb)
    g.close()
