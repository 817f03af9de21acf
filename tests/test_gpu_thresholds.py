"""The stop-threshold experiment (the paper's Fig. 3 study, sweeps and L1
distance to the fixed point against the threshold 1e-6 .. 1e-15) on R-MAT
scale 18 with edge factor 20, against the oracle: the GPU's FP64 Jacobi
sweep count at every threshold is the oracle's (+-1), every result lies
within the stop rule's bound of the oracle's fixed point, the fused sweep
needs no more sweeps than Jacobi (Sec. 5.3), and below 1e-8 both are within
1e-8 of x* in L1 (the paper's "negligible" remark)."""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import D, graph, l1

pytestmark = pytest.mark.gpu

TAUS = [10.0 ** -k for k in range(6, 16)]


def test_threshold_sweep_against_oracle():
    n, src, dst = gen.rmat(18, 20, seed=1)
    og = oracle.build_graph(n, src, dst)
    # one oracle Jacobi run gives the sweep count for every threshold (the
    # first sweep whose change is <= tau) and, continued, the fixed point
    ref = oracle.jacobi(og, D, tau=1e-15, max_iter=2000)
    hist = ref.history
    star = oracle.jacobi(og, D, tau=0.0, max_iter=len(hist) + 60).x
    g = graph(n, src, dst)
    for tau in TAUS:
        k_orc = int(np.argmax(hist <= tau)) + 1
        assert hist[k_orc - 1] <= tau
        xj, rj = g.solve(variant="jacobi", threshold=tau, max_iter=2000)
        xg, rg = g.solve(variant="gs", threshold=tau, max_iter=2000)
        assert rj.status == 0 and rg.status == 0, tau
        assert abs(rj.iters - k_orc) <= 1, (tau, rj.iters, k_orc)
        assert rg.iters <= rj.iters, (tau, rg.iters, rj.iters)
        bound = D / (1 - D) * tau + 1e-14
        assert l1(xj, star) <= bound, (tau, l1(xj, star))
        assert l1(xg, star) <= bound, (tau, l1(xg, star))
        if tau <= 1e-8:
            assert l1(xj, star) < 1e-8 and l1(xg, star) < 1e-8
    g.close()
