"""Oracle work spread over host processes (spawned, so they never inherit a
CUDA context): cancellation-free central differences of the weighted
PageRank fixed point, one edge per task.  Imports only numpy and the seeded
input generators besides the oracle."""
import numpy as np

import gen
import oracle

_state = {}


def init_weighted(scale, ef, graph_seed, weight_seed, x, grad_x, d):
    """Per worker: the same seeded weighted graph, its oracle build and row
    normalisation, the base point x and the loss gradient."""
    n, src, dst = gen.rmat(scale, ef, seed=graph_seed)
    w = gen.edge_weights(len(src), seed=weight_seed)
    og = oracle.build_graph(n, src, dst)
    _, _, csc_p = oracle.row_normalize(og, w)
    _state.update(og=og, w=w, csc_p=csc_p, x=np.asarray(x), gx=np.asarray(grad_x), d=d)


def fd_edge(e, h=1e-6):
    """(central difference of L w.r.t. raw weight e, its solve-error bound)"""
    s = _state
    return oracle.fd_weight(s["og"], s["w"], s["x"], s["gx"], int(e), h=h, d=s["d"],
                            csc_p=s["csc_p"], with_bound=True)


def fd_damping(h=1e-6):
    s = _state
    return oracle.fd_damping(s["og"], s["x"], s["gx"], h=h, d=s["d"], csc_p=s["csc_p"],
                             with_bound=True)
