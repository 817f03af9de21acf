"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no PageRank arithmetic: it draws random numbers and keeps
edge lists.  Both the CUDA library and the oracle consume what it produces;
neither imports the other.

R-MAT (Chakrabarti, Zhan, Faloutsos 2004, the Graph500 generator named in the
paper's Sec. 5.2) with a/b/c/d = 0.57/0.19/0.19/0.05, scrambled labels,
self-loops and duplicates removed.  The paper's Table 3 R-MAT rows have an
edge factor near 20; the workloads here use 16.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmat.c")
_SO = os.path.join(_HERE, "_rmat.so")
_lock = threading.Lock()
_lib = None

STREAM_WEIGHTS = 0x57474854
STREAM_SEEDS = 0x53454544
STREAM_TARGETS = 0x54415247
STREAM_COEFFS = 0x434f4546
STREAM_FD = 0x46444544
STREAM_MULTI = 0x4d554c54
STREAM_X0 = 0x58304030


def build(force: bool = False) -> str:
    """Compiles rmat.c into _rmat.so beside it (gcc, a second or two)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.gen_rmat_raw.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_int, ctypes.c_int, i32p, i32p]
            lib.gen_rmat_raw.restype = ctypes.c_int
            lib.gen_dedup.argtypes = [ctypes.c_int, ctypes.c_int64, i32p, i32p]
            lib.gen_dedup.restype = ctypes.c_int64
            lib.gen_shuffle.argtypes = [ctypes.c_int64, ctypes.c_uint64, i32p, i32p]
            lib.gen_shuffle.restype = None
            lib.gen_fix_dangling.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_uint64, i32p, i32p]
            lib.gen_fix_dangling.restype = ctypes.c_int64
            lib.gen_uniform_array.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                                              ctypes.POINTER(ctypes.c_double)]
            lib.gen_uniform_array.restype = None
            lib.gen_rand64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            lib.gen_rand64.restype = ctypes.c_uint64
            _lib = lib
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def uniform(n: int, seed: int, stream: int) -> np.ndarray:
    """n uniform doubles in [0, 1) from the counter-based generator."""
    out = np.empty(int(n), dtype=np.float64)
    _load().gen_uniform_array(int(n), int(seed), int(stream),
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, scramble: bool = True, dedup: bool = True,
         shuffle: bool = False, dangling_frac: float | None = None,
         threads: int | None = None):
    """Directed R-MAT graph with n = 2**scale vertices.

    Returns (n, src, dst) with int32 edge arrays in generation order (random).
    dangling_frac, when given, makes exactly round(frac * n) vertices dangling
    (seeded fix-up of the deduplicated graph).
    """
    lib = _load()
    n = 1 << scale
    m = int(edge_factor) * n
    extra = n if dangling_frac is not None else 0
    src = np.empty(m + extra, dtype=np.int32)
    dst = np.empty(m + extra, dtype=np.int32)
    if threads is None:
        threads = max(1, min(32, len(os.sched_getaffinity(0))))
    rc = lib.gen_rmat_raw(scale, m, a, b, c, seed, 1 if scramble else 0, threads,
                          _p32(src), _p32(dst))
    if rc != 0:
        raise ValueError("bad R-MAT parameters")
    if dedup:
        m = lib.gen_dedup(scale, m, _p32(src), _p32(dst))
        if m < 0:
            raise MemoryError("dedup failed")
    if dangling_frac is not None:
        target = int(round(dangling_frac * n))
        m = lib.gen_fix_dangling(n, m, m + extra, target, seed, _p32(src), _p32(dst))
        if m < 0:
            raise MemoryError("dangling fix-up failed")
    if shuffle:
        lib.gen_shuffle(m, seed, _p32(src), _p32(dst))
    return n, src[:m].copy(), dst[:m].copy()


# ---------------------------------------------------------------------------
# small structured graphs (closed-form and edge cases)
# ---------------------------------------------------------------------------

def cycle(n: int):
    """Directed n-cycle 0 -> 1 -> ... -> n-1 -> 0."""
    s = np.arange(n, dtype=np.int32)
    return n, s, ((s + 1) % n).astype(np.int32)


def in_star(leaves: int):
    """Leaves 1..m point at centre 0; the centre is dangling."""
    s = np.arange(1, leaves + 1, dtype=np.int32)
    return leaves + 1, s, np.zeros(leaves, dtype=np.int32)


def bi_star(leaves: int):
    """Centre 0 <-> each leaf; no dangling vertex."""
    lv = np.arange(1, leaves + 1, dtype=np.int32)
    src = np.concatenate([np.zeros(leaves, dtype=np.int32), lv])
    dst = np.concatenate([lv, np.zeros(leaves, dtype=np.int32)])
    return leaves + 1, src, dst


def complete(n: int):
    """Complete digraph without self-loops."""
    s, d = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    mask = s != d
    return n, s[mask].astype(np.int32).ravel(), d[mask].astype(np.int32).ravel()


def chain2():
    """0 -> 1, vertex 1 dangling."""
    return 2, np.array([0], dtype=np.int32), np.array([1], dtype=np.int32)


def random_digraph(n: int, p: float, seed: int, self_loops: bool = False,
                   multi: bool = False):
    """Erdos-Renyi style digraph from the counter-based generator; with multi,
    each present edge is repeated a random 1..3 times.  Edge order shuffled."""
    u = uniform(n * n * 2, seed, STREAM_X0 ^ n)
    src, dst = [], []
    for i in range(n):
        for j in range(n):
            if i == j and not self_loops:
                continue
            k = i * n + j
            if u[2 * k] < p:
                reps = 1 + int(u[2 * k + 1] * 3) if multi else 1
                src += [i] * reps
                dst += [j] * reps
    src = np.array(src, dtype=np.int32)
    dst = np.array(dst, dtype=np.int32)
    if len(src) > 1:
        order = np.argsort(uniform(len(src), seed, STREAM_X0 ^ 0x77), kind="stable")
        src, dst = src[order], dst[order]
    return n, src, dst


# ---------------------------------------------------------------------------
# workload-specific draws
# ---------------------------------------------------------------------------

def edge_weights(m: int, seed: int) -> np.ndarray:
    """Raw edge weights uniform in (0, 1] (1 - U[0,1)), float32."""
    w = (1.0 - uniform(m, seed, STREAM_WEIGHTS)).astype(np.float32)
    return np.maximum(w, np.float32(np.finfo(np.float32).tiny))


def seed_vertices(count: int, n: int, seed: int) -> np.ndarray:
    """Teleport seeds uniform in [0, n) (with replacement), int32."""
    return np.minimum((uniform(count, seed, STREAM_SEEDS) * n).astype(np.int64),
                      n - 1).astype(np.int32)


def loss_targets(count: int, n: int, seed: int):
    """`count` distinct target vertices and coefficients uniform in (-1, 1)."""
    keys = uniform(n, seed, STREAM_TARGETS)
    targets = np.argsort(keys, kind="stable")[:count].astype(np.int32)
    coeff = uniform(count, seed, STREAM_COEFFS) * 2.0 - 1.0
    return targets, coeff


def fd_edges(count: int, m: int, seed: int) -> np.ndarray:
    """Edge ids for finite-difference checks, uniform without replacement."""
    keys = uniform(m, seed, STREAM_FD)
    return np.argsort(keys, kind="stable")[:count].astype(np.int64)


def multi_graph_shapes(count: int, seed: int, scale_lo: int = 10, scale_hi: int = 18,
                       ef_lo: int = 8, ef_hi: int = 32):
    """(scale, edge_factor) pairs, each uniform on its integer range."""
    u = uniform(2 * count, seed, STREAM_MULTI)
    out = []
    for i in range(count):
        s = scale_lo + min(int(u[2 * i] * (scale_hi - scale_lo + 1)), scale_hi - scale_lo)
        ef = ef_lo + min(int(u[2 * i + 1] * (ef_hi - ef_lo + 1)), ef_hi - ef_lo)
        out.append((s, ef))
    return out


def random_x0(n: int, seed: int) -> np.ndarray:
    """Positive random start vector normalised to sum 1 (float64)."""
    x = 0.5 + uniform(n, seed, STREAM_X0)
    return x / x.sum()
