"""Pins the oracle's adjoint and gradients to complex-step derivatives of a
dense solve (no subtraction, so exact to machine precision) and its
cancellation-free central differences to the same."""
import numpy as np
import pytest

import gen
import oracle

D = 0.85


def _dense_loss_complex(n, src, dst, w, d, coeff):
    """L = coeff . x with x solving (I - d M(w)) x = (1-d)/n, in complex
    arithmetic so that Im(L(w + i h e_k)) / h is dL/dw_k (complex step)."""
    w = np.asarray(w, dtype=complex)
    s = np.zeros(n, dtype=complex)
    for e in range(len(src)):
        s[src[e]] += w[e]
    M = np.zeros((n, n), dtype=complex)
    for e in range(len(src)):
        M[dst[e], src[e]] += w[e] / s[src[e]]
    for u in range(n):
        if not any(src == u):
            M[:, u] = 1.0 / n
    A = np.eye(n) - d * M
    x = np.linalg.solve(A, np.full(n, (1 - d) / n, dtype=complex))
    return np.dot(coeff, x)


def _complex_step_grads(n, src, dst, w, d, coeff, h=1e-30):
    gw = np.empty(len(src))
    for k in range(len(src)):
        wk = np.array(w, dtype=complex)
        wk[k] += 1j * h
        gw[k] = _dense_loss_complex(n, src, dst, wk, d, coeff).imag / h
    gd = _dense_loss_complex(n, src, dst, w, d + 1j * h, coeff).imag / h
    return gw, gd


def _case(n, p, seed, weighted):
    n, src, dst = gen.random_digraph(n, p, seed=seed, multi=(seed % 2 == 0))
    w = gen.edge_weights(len(src), seed) if weighted else np.ones(len(src), np.float32)
    coeff = gen.uniform(n, seed, 99) * 2 - 1
    return n, src, dst, w, coeff


def _oracle_grads(n, src, dst, w, coeff, weighted):
    g = oracle.build_graph(n, src, dst)
    if weighted:
        s, csr_p, csc_p = oracle.row_normalize(g, w)
    else:
        csr_p = csc_p = None
    x = oracle.fixed_point(g, D, csc_p=csc_p, normalize=False).x
    lam, _, _ = oracle.adjoint(g, coeff, D, csr_p=csr_p)
    gw, gd = oracle.gradients(g, x, lam, D, w=w if weighted else None)
    return g, x, csc_p, gw, gd


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_adjoint_gradients_match_complex_step(seed, weighted):
    n, src, dst, w, coeff = _case(3 + seed, 0.45, seed, weighted)
    if len(src) == 0:
        pytest.skip("empty graph")
    g, x, csc_p, gw, gd = _oracle_grads(n, src, dst, w, coeff, weighted)
    cw, cd = _complex_step_grads(n, src, dst, w.astype(np.float64), D, coeff)
    scale = max(np.abs(cw).max(), 1e-300)
    assert np.max(np.abs(gw - cw)) <= 1e-12 * scale
    assert abs(gd - cd) <= 1e-12 * max(abs(cd), 1e-300)


def test_adjoint_solves_transposed_system():
    n, src, dst, w, coeff = _case(8, 0.3, 9, False)
    g = oracle.build_graph(n, src, dst)
    A, _ = oracle.dense_system(n, src, dst, D)
    lam, _, _ = oracle.adjoint(g, coeff, D)
    assert np.allclose(lam, np.linalg.solve(A.T, coeff), rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", [2, 3])
def test_cancellation_free_differences_match_complex_step(seed):
    n, src, dst, w, coeff = _case(7, 0.5, seed, True)
    g, x, csc_p, gw, gd = _oracle_grads(n, src, dst, w, coeff, True)
    cw, cd = _complex_step_grads(n, src, dst, w.astype(np.float64), D, coeff)
    for e in range(len(src)):
        fd = oracle.fd_weight(g, w, x, coeff, e, h=1e-6, d=D, csc_p=csc_p)
        assert abs(fd - cw[e]) <= 1e-8 * np.abs(cw).max()
    fdd = oracle.fd_damping(g, x, coeff, h=1e-6, d=D, csc_p=csc_p)
    assert abs(fdd - cd) <= 1e-8 * abs(cd)


def test_rmat_adjoint_vs_differences():
    """At R-MAT scale 10 the adjoint gradient agrees with the cancellation-free
    central differences on sampled edges to 1e-6 relative."""
    n, src, dst = gen.rmat(10, 16, seed=3)
    w = gen.edge_weights(len(src), 3)
    targets, c = gen.loss_targets(50, n, 3)
    coeff = np.zeros(n)
    coeff[targets] = c
    g, x, csc_p, gw, gd = _oracle_grads(n, src, dst, w, coeff, True)
    edges = gen.fd_edges(8, len(src), 3)
    fd = np.array([oracle.fd_weight(g, w, x, coeff, int(e), h=1e-6, d=D, csc_p=csc_p)
                   for e in edges])
    assert np.linalg.norm(fd - gw[edges]) <= 1e-6 * np.linalg.norm(gw[edges])
    fdd = oracle.fd_damping(g, x, coeff, h=1e-6, d=D, csc_p=csc_p)
    assert abs(fdd - gd) <= 1e-6 * abs(gd)
