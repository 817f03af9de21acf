"""Helpers shared by the GPU parity tests."""
import numpy as np
import torch

D = 0.85
BOUND = D / (1 - D) * 1e-10  # ||x - x*||_1 after a stop at L1 successive difference 1e-10


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def graph(n, src, dst, w=None, **kw):
    import paper_2203_09284_gb300 as fp
    return fp.Graph(n, dev(src), dev(dst), None if w is None else dev(w), **kw)


def l1(a, b):
    a = a.cpu().numpy() if isinstance(a, torch.Tensor) else a
    b = b.cpu().numpy() if isinstance(b, torch.Tensor) else b
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).sum())


def top_order_matches(x, xstar, k=100, bound=BOUND):
    """Orders by (rank desc, id asc); inversions are allowed only between
    vertices whose x* ranks differ by less than twice the error bound."""
    x = np.asarray(x)
    n = len(x)
    k = min(k, n)
    ids = np.arange(n)
    top_g = np.lexsort((ids, -x))[:k]
    top_s = np.lexsort((ids, -xstar))[:k]
    if np.array_equal(top_g, top_s):
        return True
    # every vertex in one list but not the other must be a near tie at the cut
    cut = xstar[top_s[-1]]
    for v in set(top_g) ^ set(top_s):
        if abs(xstar[v] - cut) >= 2 * bound:
            return False
    pos = {v: i for i, v in enumerate(top_s)}
    common = [v for v in top_g if v in pos]
    for i in range(len(common)):
        for j in range(i + 1, len(common)):
            a, b = common[i], common[j]
            if pos[a] > pos[b] and abs(xstar[a] - xstar[b]) >= 2 * bound:
                return False
    return True
