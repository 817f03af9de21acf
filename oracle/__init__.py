"""CPU oracle for the fused PageRank path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded FP64 implementation (``oracle.c``) of what the
CUDA library computes, wrapped with ctypes.  Only the tests, the smoke check
and the benchmark's CPU-baseline leg may import this package; the library
itself never does, and the two share no code.

Functions follow the paper: Algorithm 1 / Eq. 2 (Jacobi, ``jacobi``),
Algorithm 2 / Eq. 9 (sequential fused Gauss-Seidel, ``gauss_seidel``), the
Sec. 3 storage layout (``build``), plus the adjoint and gradients of the
fixed point and dense solves for tiny graphs.  All are pinned by the CPU test
suite against closed forms, numpy, complex-step derivatives and exact
rational arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_OOM, NOT_CONVERGED = 0, 1, 2, 4
NORM_L1, NORM_LINF = 0, 1


def build(force: bool = False) -> str:
    """Compiles oracle.c (plain C, no contraction of multiply-adds)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_I32 = ctypes.POINTER(ctypes.c_int32)
_F64 = ctypes.POINTER(ctypes.c_double)
_F32 = ctypes.POINTER(ctypes.c_float)
_PROBLEM = [ctypes.c_int32, _I32, _I32, _I32, _F64, _F64, ctypes.c_double, _F64, _F64,
            ctypes.c_int32]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.orc_build.argtypes = [ctypes.c_int32, ctypes.c_int64, _I32, _I32, _I32, _I32,
                                      _I32, _I32, _I32, _I32, _I32, _I32, _F64]
            lib.orc_relabel.argtypes = [ctypes.c_int32, ctypes.c_int64, _I32, _I32, _I32, _I32,
                                        _I32, _I32, _I32]
            lib.orc_bins.argtypes = [ctypes.c_int32, _I32, ctypes.c_int32, ctypes.c_int32,
                                     _I32, _I32, _I32, _I32]
            lib.orc_bins.restype = None
            it = [_F64, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _F64,
                  _I32, _F64, _F64, _F64]
            lib.orc_jacobi.argtypes = _PROBLEM + it
            lib.orc_gauss_seidel.argtypes = _PROBLEM + [ctypes.c_int32] + it
            lib.orc_perforated.argtypes = _PROBLEM + [ctypes.c_double, ctypes.c_int32] + it + [
                ctypes.POINTER(ctypes.c_int64)]
            lib.orc_fixed_point.argtypes = _PROBLEM + [_F64, ctypes.c_double, ctypes.c_int32,
                                                       ctypes.c_int32, ctypes.c_int32, _F64,
                                                       _I32, _F64, _F64]
            lib.orc_row_normalize.argtypes = [ctypes.c_int32, ctypes.c_int64, _I32, _I32, _I32,
                                              _I32, _F32, _F64, _F64, _F64]
            lib.orc_adjoint.argtypes = [ctypes.c_int32, _I32, _I32, _I32, _F64, _F64,
                                        ctypes.c_double, _F64, ctypes.c_double, ctypes.c_int32,
                                        ctypes.c_int32, _F64, _I32, _F64]
            lib.orc_gradients.argtypes = [ctypes.c_int32, ctypes.c_int64, _I32, _I32, _I32, _I32,
                                          _F32, ctypes.c_double, _F64, _F64, _F64, _F64]
            lib.orc_dense_system.argtypes = [ctypes.c_int32, ctypes.c_int64, _I32, _I32, _F64,
                                             ctypes.c_double, _F64, ctypes.c_int32, _F64, _F64]
            lib.orc_dense_solve.argtypes = [ctypes.c_int32, _F64, _F64, _F64]
            _lib = lib
    return _lib


def _p(a, t):
    if a is None:
        return ctypes.cast(None, t)
    return a.ctypes.data_as(t)


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Graph:
    """Oracle build of an edge list (Sec. 3 storage)."""
    n: int
    m: int
    src: np.ndarray
    dst: np.ndarray
    outdeg: np.ndarray
    indeg: np.ndarray
    row_ptr: np.ndarray
    col_idx: np.ndarray
    csr_eid: np.ndarray
    col_ptr: np.ndarray
    row_idx: np.ndarray
    csc_eid: np.ndarray
    inv_outdeg: np.ndarray

    def offset_list(self) -> np.ndarray:
        """For each out-list slot, the in-list slot of the same edge (the
        paper's offsetList pointing into its contributionList)."""
        pos = np.empty(self.m, dtype=np.int64)
        pos[self.csc_eid] = np.arange(self.m)
        return pos[self.csr_eid]


def build_graph(n: int, src, dst) -> Graph:
    """Degrees, CSR (out-lists by (dst, id)), CSC (in-lists by (src, id)),
    inv_outdeg = 1/outdeg (0 for dangling)."""
    lib = _load()
    src, dst = _i32(src), _i32(dst)
    m = len(src)
    outdeg = np.empty(n, np.int32)
    indeg = np.empty(n, np.int32)
    row_ptr = np.empty(n + 1, np.int32)
    col_ptr = np.empty(n + 1, np.int32)
    col_idx = np.empty(max(m, 1), np.int32)
    csr_eid = np.empty(max(m, 1), np.int32)
    row_idx = np.empty(max(m, 1), np.int32)
    csc_eid = np.empty(max(m, 1), np.int32)
    inv = np.empty(n, np.float64)
    rc = lib.orc_build(n, m, _p(src, _I32), _p(dst, _I32), _p(outdeg, _I32), _p(indeg, _I32),
                       _p(row_ptr, _I32), _p(col_idx, _I32), _p(csr_eid, _I32),
                       _p(col_ptr, _I32), _p(row_idx, _I32), _p(csc_eid, _I32), _p(inv, _F64))
    if rc != OK:
        raise ValueError(f"orc_build failed ({rc})")
    return Graph(n, m, src, dst, outdeg, indeg, row_ptr, col_idx[:m], csr_eid[:m], col_ptr,
                 row_idx[:m], csc_eid[:m], inv)


def relabel(g: Graph):
    """Degree-ordered relabelling: new_to_old (in-degree descending, ties by
    id) and the in-lists in the new ids (rcol_ptr, rrow_idx, rcsc_eid)."""
    lib = _load()
    n2o = np.empty(g.n, np.int32)
    rcol = np.empty(g.n + 1, np.int32)
    rrow = np.empty(max(g.m, 1), np.int32)
    reid = np.empty(max(g.m, 1), np.int32)
    rc = lib.orc_relabel(g.n, g.m, _p(g.src, _I32), _p(g.dst, _I32), _p(g.indeg, _I32),
                         _p(n2o, _I32), _p(rcol, _I32), _p(rrow, _I32), _p(reid, _I32))
    if rc != OK:
        raise ValueError(f"orc_relabel failed ({rc})")
    return n2o, rcol, rrow[:g.m], reid[:g.m]


def bins(g: Graph, t_lo: int, t_hub: int):
    lib = _load()
    low = np.empty(g.n, np.int32)
    mid = np.empty(g.n, np.int32)
    hub = np.empty(g.n, np.int32)
    cnt = np.empty(3, np.int32)
    lib.orc_bins(g.n, _p(g.indeg, _I32), t_lo, t_hub, _p(low, _I32), _p(mid, _I32),
                 _p(hub, _I32), _p(cnt, _I32))
    return low[:cnt[0]].copy(), mid[:cnt[1]].copy(), hub[:cnt[2]].copy()


@dataclass
class Result:
    x: np.ndarray
    iters: int
    err: float
    history: np.ndarray
    sum_before: float
    status: int


def _problem(g: Graph, d, csc_p=None, tele=None, rhs=None, dangling_along_tele=False):
    csc_p, tele, rhs = _f64(csc_p), _f64(tele), _f64(rhs)
    keep = (csc_p, tele, rhs)
    args = [g.n, _p(g.col_ptr, _I32), _p(g.row_idx, _I32), _p(g.outdeg, _I32),
            _p(g.inv_outdeg, _F64), _p(csc_p, _F64), float(d), _p(tele, _F64), _p(rhs, _F64),
            1 if dangling_along_tele else 0]
    return args, keep


def _iterate(fn, g, d, tau, max_iter, norm, normalize, x0, pre=(), **kw):
    args, keep = _problem(g, d, **kw)
    args = args + list(pre)
    x0 = _f64(x0)
    x = np.empty(g.n, np.float64)
    hist = np.zeros(max(max_iter, 1), np.float64)
    iters = ctypes.c_int32(0)
    err = ctypes.c_double(0)
    sb = ctypes.c_double(0)
    rc = fn(*args, _p(x0, _F64), float(tau), int(max_iter), int(norm), 1 if normalize else 0,
            _p(x, _F64), ctypes.byref(iters), ctypes.byref(err), _p(hist, _F64), ctypes.byref(sb))
    del keep
    if rc not in (OK, NOT_CONVERGED):
        raise ValueError(f"oracle iteration failed ({rc})")
    return Result(x, iters.value, err.value, hist[:iters.value].copy(), sb.value, rc)


def jacobi(g: Graph, d=0.85, tau=1e-10, max_iter=200, norm=NORM_L1, normalize=True, x0=None,
           **kw) -> Result:
    """Algorithm 1 with uniform dangling mass (or a teleport / right-hand side)."""
    return _iterate(_load().orc_jacobi, g, d, tau, max_iter, norm, normalize, x0, **kw)


def gauss_seidel(g: Graph, d=0.85, tau=1e-10, max_iter=200, norm=NORM_L1, normalize=True,
                 x0=None, renorm=True, **kw) -> Result:
    """Algorithm 2 / Eq. 9 in increasing vertex id order; with renorm each
    sweep ends with x /= sum x (the sum drifts under in-place updates)."""
    return _iterate(_load().orc_gauss_seidel, g, d, tau, max_iter, norm, normalize, x0,
                    pre=(1 if renorm else 0,), **kw)


@dataclass
class PerforatedResult(Result):
    gathered: int = 0


def perforated(g: Graph, d=0.85, eps=1e-8, period=0, tau=1e-10, max_iter=200, norm=NORM_L1,
               normalize=True, x0=None, **kw) -> PerforatedResult:
    """Loop-perforated Jacobi: in a perforated sweep a vertex whose last
    change was below eps times its value keeps it (no in-list sum).  With
    period > 0 every period-th sweep is full and only those stop; with period
    0 any sweep stops.  ``gathered`` = in-list entries summed in all sweeps."""
    lib = _load()
    args, keep = _problem(g, d, **kw)
    x0 = _f64(x0)
    x = np.empty(g.n, np.float64)
    hist = np.zeros(max(max_iter, 1), np.float64)
    iters = ctypes.c_int32(0)
    err = ctypes.c_double(0)
    sb = ctypes.c_double(0)
    gathered = ctypes.c_int64(0)
    rc = lib.orc_perforated(*args, float(eps), int(period), _p(x0, _F64), float(tau),
                            int(max_iter), int(norm), 1 if normalize else 0, _p(x, _F64),
                            ctypes.byref(iters), ctypes.byref(err), _p(hist, _F64),
                            ctypes.byref(sb), ctypes.byref(gathered))
    del keep
    if rc not in (OK, NOT_CONVERGED):
        raise ValueError(f"orc_perforated failed ({rc})")
    return PerforatedResult(x, iters.value, err.value, hist[:iters.value].copy(), sb.value, rc,
                            gathered.value)


def fixed_point(g: Graph, d=0.85, x0=None, floor_tau=0.0, patience=5, max_iter=5000,
                normalize=True, **kw) -> Result:
    """Tight Jacobi fixed point (to round-off stagnation).  ``err`` is the last
    L1 successive difference; ||x - x*||_1 <= d/(1-d) * err."""
    lib = _load()
    args, keep = _problem(g, d, **kw)
    x0 = _f64(x0)
    x = np.empty(g.n, np.float64)
    iters = ctypes.c_int32(0)
    err = ctypes.c_double(0)
    sb = ctypes.c_double(0)
    rc = lib.orc_fixed_point(*args, _p(x0, _F64), float(floor_tau), int(patience), int(max_iter),
                             1 if normalize else 0, _p(x, _F64), ctypes.byref(iters),
                             ctypes.byref(err), ctypes.byref(sb))
    del keep
    if rc != OK:
        raise ValueError(f"orc_fixed_point failed ({rc})")
    return Result(x, iters.value, err.value, np.zeros(0), sb.value, rc)


def row_normalize(g: Graph, w):
    """Row sums s_u of raw weights (out-list order) and P per CSR / CSC slot."""
    lib = _load()
    w = np.ascontiguousarray(w, dtype=np.float32)
    s = np.empty(g.n, np.float64)
    csr_p = np.empty(max(g.m, 1), np.float64)
    csc_p = np.empty(max(g.m, 1), np.float64)
    lib.orc_row_normalize(g.n, g.m, _p(g.row_ptr, _I32), _p(g.csr_eid, _I32),
                          _p(g.csc_eid, _I32), _p(g.row_idx, _I32), _p(w, _F32), _p(s, _F64),
                          _p(csr_p, _F64), _p(csc_p, _F64))
    return s, csr_p[:g.m], csc_p[:g.m]


def adjoint(g: Graph, grad_x, d=0.85, csr_p=None, floor_tau=0.0, patience=5, max_iter=5000):
    """lambda solving (I - d M)^T lambda = grad_x, iterated over the out-lists."""
    lib = _load()
    gx = _f64(grad_x)
    csr_p = _f64(csr_p)
    lam = np.empty(g.n, np.float64)
    iters = ctypes.c_int32(0)
    err = ctypes.c_double(0)
    rc = lib.orc_adjoint(g.n, _p(g.row_ptr, _I32), _p(g.col_idx, _I32), _p(g.outdeg, _I32),
                         _p(g.inv_outdeg, _F64), _p(csr_p, _F64), float(d), _p(gx, _F64),
                         float(floor_tau), int(patience), int(max_iter), _p(lam, _F64),
                         ctypes.byref(iters), ctypes.byref(err))
    if rc != OK:
        raise ValueError(f"orc_adjoint failed ({rc})")
    return lam, iters.value, err.value


def gradients(g: Graph, x, lam, d=0.85, w=None):
    """(dL/dw in input edge order, dL/dd) from the fixed point and adjoint."""
    lib = _load()
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    x, lam = _f64(x), _f64(lam)
    gw = np.zeros(max(g.m, 1), np.float64)
    gd = ctypes.c_double(0)
    rc = lib.orc_gradients(g.n, g.m, _p(g.row_ptr, _I32), _p(g.col_idx, _I32),
                           _p(g.csr_eid, _I32), _p(g.outdeg, _I32), _p(w, _F32), float(d),
                           _p(x, _F64), _p(lam, _F64), _p(gw, _F64), ctypes.byref(gd))
    if rc != OK:
        raise ValueError(f"orc_gradients failed ({rc})")
    return gw[:g.m], gd.value


def dense_system(n, src, dst, d=0.85, w=None, tele=None, dangling_along_tele=False):
    """A = I - d M and b = (1-d) v for a tiny graph (row-major)."""
    lib = _load()
    src, dst = _i32(src), _i32(dst)
    w, tele = _f64(w), _f64(tele)
    A = np.empty((n, n), np.float64)
    b = np.empty(n, np.float64)
    lib.orc_dense_system(n, len(src), _p(src, _I32), _p(dst, _I32), _p(w, _F64), float(d),
                         _p(tele, _F64), 1 if dangling_along_tele else 0, _p(A, _F64),
                         _p(b, _F64))
    return A, b


def dense_solve(A, b):
    """Gaussian elimination with partial pivoting (copies its inputs)."""
    lib = _load()
    A = np.array(A, dtype=np.float64, order="C")
    b = np.array(b, dtype=np.float64)
    n = len(b)
    x = np.empty(n, np.float64)
    rc = lib.orc_dense_solve(n, _p(A, _F64), _p(b, _F64), _p(x, _F64))
    if rc != OK:
        raise ValueError("singular system")
    return x


def dense_pagerank(n, src, dst, d=0.85, w=None, tele=None, dangling_along_tele=False):
    A, b = dense_system(n, src, dst, d, w, tele, dangling_along_tele)
    return dense_solve(A, b)


# ---------------------------------------------------------------------------
# Cancellation-free central differences (composition of the routines above)
# ---------------------------------------------------------------------------

def _out_edges(g: Graph, eid):
    """Source u of edge eid, u's out-edges (input ids, out-list order) and,
    for every edge, its in-list slot."""
    u = int(g.src[eid])
    out_ids = g.csr_eid[int(g.row_ptr[u]):int(g.row_ptr[u + 1])]
    pos = np.empty(g.m, dtype=np.int64)
    pos[g.csc_eid] = np.arange(g.m)
    return u, out_ids, pos


def fd_weight(g: Graph, w, x, grad_x, eid, h=1e-6, d=0.85, csc_p=None, with_bound=False):
    """Central difference of L = grad_x . x* w.r.t. raw weight w[eid], computed
    as g^T (x(w+h) - x(w-h)) / 2h where each half-difference is solved directly:
      (I - d M+) (x+ - x) = d (M+ - M) x,   (I - d M-) (x - x-) = d (M - M-) x.
    The right-hand sides live on the out-neighbours of the edge's source, so
    there is no subtraction of two nearly equal solutions.
    With with_bound, also returns a bound on the error the two stopped solves
    leave in the result: each stops at an L1 change `err`, so its solution is
    within d/(1-d) err of the exact one in L1 (d M is a 1-norm contraction
    by d), and the quotient is off by at most |grad_x|_inf times their sum /
    2h."""
    if csc_p is None:
        _, _, csc_p = row_normalize(g, w)
    total = np.zeros(g.n)
    solve_err = 0.0
    u, out_ids, pos = _out_edges(g, eid)
    wf = [float(np.float64(np.float32(w[e]))) for e in out_ids]
    s0 = 0.0
    for we in wf:  # out-list order, like orc_row_normalize
        s0 += we
    for sign in (+1.0, -1.0):
        # raw weight w_e + delta: u's row sum becomes s0 + delta, and the
        # change of each P_uv' is written without subtracting two nearly
        # equal quotients:
        #   (w_e + delta)/(s0 + delta) - w_e/s0 = delta (s0 - w_e) / (s0 s1)
        #   w_e'/(s0 + delta) - w_e'/s0        = -w_e' delta / (s0 s1)
        delta = sign * h
        q = delta / (s0 * (s0 + delta))
        p2 = np.array(csc_p, dtype=np.float64)
        rhs = np.zeros(g.n)
        for e, we in zip(out_ids, wf):
            v = int(g.dst[e])
            diff = q * (s0 - we) if int(e) == int(eid) else -we * q
            p2[pos[e]] = we / s0 + diff
            rhs[v] += d * x[u] * diff * sign
        tau = 1e-13 * np.abs(rhs).sum()
        r = fixed_point(g, d, x0=np.zeros(g.n), floor_tau=tau, patience=5, normalize=False,
                        csc_p=p2, rhs=rhs)
        total += r.x
        solve_err += d / (1.0 - d) * r.err
    fd = float(np.dot(grad_x, total) / (2.0 * h))
    if with_bound:
        return fd, float(np.abs(grad_x).max() * solve_err / (2.0 * h))
    return fd


def fd_damping(g: Graph, x, grad_x, h=1e-6, d=0.85, csc_p=None, with_bound=False):
    """Central difference of L w.r.t. d with the same direct difference solves:
      (I - (d+h) M)(x+ - x) = h (M x - 1/n),  (I - (d-h) M)(x - x-) = h (M x - 1/n)."""
    n = g.n
    # M x = P^T x + D/n, computed here from one un-damped Jacobi sweep:
    # with d = 1 and r = 0 the sweep returns exactly M x.
    mx = jacobi(g, d=1.0, tau=-1.0, max_iter=1, normalize=False, x0=x, csc_p=csc_p,
                rhs=np.zeros(n)).x
    rhs = h * (mx - 1.0 / n)
    tau = 1e-13 * np.abs(rhs).sum()
    total = np.zeros(n)
    solve_err = 0.0
    for dd in (d + h, d - h):
        r = fixed_point(g, dd, x0=np.zeros(n), floor_tau=tau, patience=5, normalize=False,
                        csc_p=csc_p, rhs=rhs)
        total += r.x
        solve_err += dd / (1.0 - dd) * r.err
    fd = float(np.dot(grad_x, total) / (2.0 * h))
    if with_bound:
        return fd, float(np.abs(grad_x).max() * solve_err / (2.0 * h))
    return fd
