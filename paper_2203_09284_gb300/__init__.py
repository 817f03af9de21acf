"""GB300-native fused PageRank (FusEd-PageRank, arXiv 2203.09284).

Thin ctypes binding of ``libfusedpr.so`` (C ABI in ``include/fusedpr.h``).
Functions keep the C names (``pr_graph_create``, ``pr_solve``, ...); this
module only marshals arguments.  Every step of the computation runs in the
library's CUDA kernels; PyTorch provides device memory (tensors and its caching
allocator) and streams.  There is no CPU fallback: importing works without a
GPU, but every call needs the built library and a CUDA device.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _build

__all__ = [
    "PR_OK", "PR_ERR_INVALID_ARG", "PR_ERR_OOM", "PR_ERR_CUDA", "PR_NOT_CONVERGED",
    "PR_ERR_TIMEOUT", "PR_ERR_UNSUPPORTED", "PR_ERR_NUMERIC", "PR_JACOBI", "PR_FUSED_GS", "PR_FP64", "PR_FP32",
    "PR_FP32_DC", "PR_BF16_DC", "PR_FP16_DC", "PR_NORM_L1", "PR_NORM_LINF", "PR_BUILD_CSR",
    "PR_DEDUP",
    "PrOptions", "PrResult", "PrTune", "PrAllocator", "PageRankError", "lib", "library_path",
    "pr_options_default", "pr_graph_create", "pr_graph_destroy", "pr_graph_info",
    "pr_graph_export", "pr_solve", "pr_solve_batched", "pr_solve_multi", "pr_backward",
    "pr_scan_exclusive_noalloc", "pr_gather_probe", "pr_status_string", "pr_last_error", "pr_kernel_launches", "Graph",
]

PR_OK, PR_ERR_INVALID_ARG, PR_ERR_OOM, PR_ERR_CUDA = 0, 1, 2, 3
PR_NOT_CONVERGED, PR_ERR_TIMEOUT, PR_ERR_UNSUPPORTED, PR_ERR_NUMERIC = 4, 5, 6, 7
PR_JACOBI, PR_FUSED_GS = 0, 1
PR_FP64, PR_FP32, PR_FP32_DC, PR_BF16_DC, PR_FP16_DC = 0, 1, 2, 3, 4
PR_NORM_L1, PR_NORM_LINF = 0, 1
PR_BUILD_CSR = 1
PR_DEDUP = 2

VARIANTS = {"jacobi": PR_JACOBI, "gs": PR_FUSED_GS, "fused_gs": PR_FUSED_GS}
PRECISIONS = {"fp64": PR_FP64, "fp32": PR_FP32, "fp32_dc": PR_FP32_DC, "bf16_dc": PR_BF16_DC,
              "fp16_dc": PR_FP16_DC}
NORMS = {"l1": PR_NORM_L1, "linf": PR_NORM_LINF}


class PrTune(ctypes.Structure):
    _fields_ = [("t_lo", ctypes.c_int32), ("t_hub", ctypes.c_int32), ("hub_seg", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("deterministic_gs", ctypes.c_int32),
                ("stage_kb", ctypes.c_int32), ("wait_limit", ctypes.c_int32),
                ("fused_split", ctypes.c_int32), ("mid_wide", ctypes.c_int32),
                ("blocking", ctypes.c_int32)]


class PrOptions(ctypes.Structure):
    _fields_ = [("d", ctypes.c_double), ("threshold", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("variant", ctypes.c_int),
                ("precision", ctypes.c_int), ("norm", ctypes.c_int),
                ("x0", ctypes.c_void_p), ("history", ctypes.c_void_p),
                ("use_graph", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("inner_rel", ctypes.c_double), ("tune", ctypes.POINTER(PrTune)),
                ("no_rescale", ctypes.c_int32), ("perforate_eps", ctypes.c_double),
                ("perforate_period", ctypes.c_int32)]


class PrResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer_iters", ctypes.c_int32),
                ("residual", ctypes.c_double), ("sum_before_norm", ctypes.c_double),
                ("status", ctypes.c_int), ("gathered", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                            ctypes.c_void_p)


class PrAllocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


class PageRankError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = pr_status_string(status)
        detail = pr_last_error()
        super().__init__(f"{where}: {msg}" + (f" ({detail})" if detail else ""))


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.OUT


def lib():
    """The loaded libfusedpr.so.  Raises if it has not been built: there is no
    fallback path."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.OUT):
                raise RuntimeError(
                    f"{_build.OUT} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback)")
            L = ctypes.CDLL(_build.OUT)
            vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            L.pr_options_default.argtypes = [ctypes.POINTER(PrOptions)]
            L.pr_graph_create.argtypes = [i32, i64, vp, vp, vp, ctypes.c_uint32,
                                          ctypes.POINTER(PrAllocator), vp,
                                          ctypes.POINTER(ctypes.c_void_p)]
            L.pr_graph_destroy.argtypes = [vp]
            L.pr_graph_destroy.restype = None
            L.pr_graph_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64),
                                        ctypes.POINTER(i32), ctypes.POINTER(i32)]
            L.pr_graph_export.argtypes = [vp] + [vp] * 12 + [vp]
            L.pr_solve.argtypes = [vp, ctypes.POINTER(PrOptions), vp, ctypes.POINTER(PrResult), vp]
            L.pr_solve_batched.argtypes = [vp, ctypes.POINTER(PrOptions), i32, vp, vp, vp,
                                           ctypes.POINTER(PrResult), vp]
            L.pr_solve_multi.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(PrOptions),
                                         ctypes.POINTER(vp), ctypes.POINTER(PrResult), vp]
            L.pr_backward.argtypes = [vp, ctypes.POINTER(PrOptions), vp, vp, vp, vp,
                                      ctypes.POINTER(PrResult), vp]
            L.pr_scan_exclusive_noalloc.argtypes = [vp, vp, i64, vp]
            L.pr_gather_probe.argtypes = [vp, i64, vp, i32, i32, vp, vp]
            L.pr_status_string.argtypes = [ctypes.c_int]
            L.pr_status_string.restype = ctypes.c_char_p
            L.pr_last_error.argtypes = []
            L.pr_last_error.restype = ctypes.c_char_p
            L.pr_kernel_launches.argtypes = []
            L.pr_kernel_launches.restype = ctypes.c_uint64
            for name in ("pr_options_default", "pr_graph_create", "pr_graph_info",
                         "pr_graph_export", "pr_solve", "pr_solve_batched", "pr_solve_multi",
                         "pr_backward", "pr_scan_exclusive_noalloc", "pr_gather_probe"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


# ---------------------------------------------------------------------------
# C names, argument marshalling only
# ---------------------------------------------------------------------------

def pr_status_string(status: int) -> str:
    return lib().pr_status_string(int(status)).decode()


def pr_last_error() -> str:
    return lib().pr_last_error().decode()


def pr_kernel_launches() -> int:
    return int(lib().pr_kernel_launches())


kernel_launches = pr_kernel_launches


def pr_options_default() -> PrOptions:
    o = PrOptions()
    lib().pr_options_default(ctypes.byref(o))
    return o


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(status, where, ok=(PR_OK,)):
    if status not in ok:
        raise PageRankError(status, where)
    return status


# torch caching-allocator hooks (kept alive for the process lifetime)
def _torch_alloc(nbytes, stream, ctx):
    try:
        dev = torch.cuda.current_device()
        return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
    except Exception:  # out of memory: the library reports PR_ERR_OOM
        return None


def _torch_free(ptr, nbytes, stream, ctx):
    torch.cuda.caching_allocator_delete(ptr)


_TORCH_ALLOCATOR = PrAllocator(_ALLOC_FN(_torch_alloc), _FREE_FN(_torch_free), None)


def torch_allocator() -> PrAllocator:
    """Allocator hooks that route library allocations through torch's caching
    allocator."""
    return _TORCH_ALLOCATOR


def _device_readable(t):
    return t.is_cuda or (t.device.type == "cpu" and t.is_pinned())


def pr_graph_create(n, src, dst, w=None, flags=0, allocator=None, stream=None):
    """Builds a graph from int32 tensors src/dst (and optional float32
    weights) on the device or in pinned host memory (read once by the build,
    no separate copy).  Returns an opaque handle (int)."""
    for t, name in ((src, "src"), (dst, "dst")):
        if not (_device_readable(t) and t.dtype == torch.int32 and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous int32 CUDA or pinned host tensor")
    if w is not None and not (_device_readable(w) and w.dtype == torch.float32
                              and w.is_contiguous()):
        raise ValueError("w must be a contiguous float32 CUDA or pinned host tensor")
    out = ctypes.c_void_p()
    alloc = ctypes.byref(allocator) if allocator is not None else None
    st = lib().pr_graph_create(int(n), int(src.numel()), _ptr(src), _ptr(dst), _ptr(w),
                               int(flags), alloc, _stream(stream), ctypes.byref(out))
    _check(st, "pr_graph_create")
    return out.value


def pr_graph_destroy(handle):
    if handle:
        lib().pr_graph_destroy(ctypes.c_void_p(handle))


def pr_graph_info(handle):
    n, m, nd = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    bins = (ctypes.c_int32 * 3)()
    _check(lib().pr_graph_info(ctypes.c_void_p(handle), ctypes.byref(n), ctypes.byref(m),
                               ctypes.byref(nd), bins), "pr_graph_info")
    return {"n": n.value, "m": m.value, "n_dangling": nd.value, "bins": list(bins)}


def pr_graph_export(handle, stream=None, csr=False):
    """Copies the build products into new device tensors (dict)."""
    info = pr_graph_info(handle)
    n, m = info["n"], info["m"]
    dev = torch.device("cuda", torch.cuda.current_device())
    i32 = dict(dtype=torch.int32, device=dev)
    out = {
        "outdeg": torch.empty(n, **i32), "indeg": torch.empty(n, **i32),
        "col_ptr": torch.empty(n + 1, **i32), "row_idx": torch.empty(m, **i32),
        "csc_eid": torch.empty(m, **i32), "inv_outdeg": torch.empty(n, dtype=torch.float64,
                                                                    device=dev),
        "new_to_old": torch.empty(n, **i32), "rcol_ptr": torch.empty(n + 1, **i32),
        "rrow_idx": torch.empty(m, **i32),
    }
    if csr:
        out.update(row_ptr=torch.empty(n + 1, **i32), col_idx=torch.empty(m, **i32),
                   csr_eid=torch.empty(m, **i32))
    g = out.get
    st = lib().pr_graph_export(ctypes.c_void_p(handle), _ptr(g("outdeg")), _ptr(g("indeg")),
                               _ptr(g("col_ptr")), _ptr(g("row_idx")), _ptr(g("csc_eid")),
                               _ptr(g("row_ptr")), _ptr(g("col_idx")), _ptr(g("csr_eid")),
                               _ptr(g("inv_outdeg")), _ptr(g("new_to_old")),
                               _ptr(g("rcol_ptr")), _ptr(g("rrow_idx")), _stream(stream))
    _check(st, "pr_graph_export")
    return out


def make_options(d=0.85, threshold=1e-10, max_iter=1000, variant="jacobi", precision="fp64",
                 norm="l1", x0=None, history=None, use_graph=True, max_outer=0, inner_rel=0.0,
                 tune=None, no_rescale=False, perforate_eps=0.0, perforate_period=0):
    o = pr_options_default()
    o.d, o.threshold, o.max_iter = float(d), float(threshold), int(max_iter)
    o.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.norm = NORMS[norm] if isinstance(norm, str) else int(norm)
    o.x0 = x0.data_ptr() if x0 is not None else None
    o.history = history.data_ptr() if history is not None else None
    o.use_graph = 1 if use_graph else 0
    o.max_outer = int(max_outer)
    o.inner_rel = float(inner_rel)
    o.no_rescale = 1 if no_rescale else 0
    o.perforate_eps = float(perforate_eps)
    o.perforate_period = int(perforate_period)
    if tune is not None:
        t = tune if isinstance(tune, PrTune) else PrTune(**tune)
        o._tune_ref = t
        o.tune = ctypes.pointer(t)
    return o


def pr_solve(handle, options, x_out, stream=None):
    """Solves into x_out (float64 device tensor [n]); returns PrResult."""
    r = PrResult()
    st = lib().pr_solve(ctypes.c_void_p(handle), ctypes.byref(options), _ptr(x_out),
                        ctypes.byref(r), _stream(stream))
    _check(st, "pr_solve", ok=(PR_OK, PR_NOT_CONVERGED))
    return r


def pr_solve_batched(handle, options, seeds, X_out, stream=None, V=None):
    """Personalised PageRank of B columns: one-hot seeds (int32 [B]) or dense
    teleport vectors V ([n][B], X_out's type); returns B PrResults."""
    B = int(seeds.numel()) if seeds is not None else int(V.shape[1])
    res = (PrResult * max(B, 1))()
    st = lib().pr_solve_batched(ctypes.c_void_p(handle), ctypes.byref(options), B, _ptr(seeds),
                                _ptr(V), _ptr(X_out), res, _stream(stream))
    _check(st, "pr_solve_batched", ok=(PR_OK, PR_NOT_CONVERGED))
    return list(res)[:B]


def pr_solve_multi(handles, options, x_outs, stream=None):
    G = len(handles)
    harr = (ctypes.c_void_p * G)(*[ctypes.c_void_p(h) for h in handles])
    xarr = (ctypes.c_void_p * G)(*[ctypes.c_void_p(x.data_ptr()) for x in x_outs])
    res = (PrResult * G)()
    st = lib().pr_solve_multi(harr, G, ctypes.byref(options), xarr, res, _stream(stream))
    _check(st, "pr_solve_multi", ok=(PR_OK, PR_NOT_CONVERGED))
    return list(res)


def pr_scan_exclusive_noalloc(inp, out, count=None, stream=None):
    """out[0..count] = exclusive prefix sums of inp[0..count) (int32 device
    tensors), using the library's fixed scratch array (no allocation)."""
    count = int(inp.numel()) if count is None else int(count)
    st = lib().pr_scan_exclusive_noalloc(_ptr(inp), _ptr(out), count, _stream(stream))
    _check(st, "pr_scan_exclusive_noalloc")


def pr_gather_probe(idx, y, sink, hot=0, stream=None):
    """sink += sum of y[idx] with the sweep's gather pattern (diagnostic)."""
    st = lib().pr_gather_probe(_ptr(idx), int(idx.numel()), _ptr(y), int(y.numel()), int(hot),
                               _ptr(sink), _stream(stream))
    _check(st, "pr_gather_probe")


def pr_backward(handle, options, x, grad_x, grad_w=None, grad_d=None, stream=None):
    r = PrResult()
    st = lib().pr_backward(ctypes.c_void_p(handle), ctypes.byref(options), _ptr(x), _ptr(grad_x),
                           _ptr(grad_w), _ptr(grad_d), ctypes.byref(r), _stream(stream))
    _check(st, "pr_backward", ok=(PR_OK, PR_NOT_CONVERGED))
    return r


class Graph:
    """Owns a pr_graph handle built from edge tensors on the device or in
    pinned host memory."""

    def __init__(self, n, src, dst, w=None, build_csr=False, use_torch_allocator=True,
                 stream=None, dedup=False):
        self.n = int(n)
        self.m = int(src.numel())  # input edges (pr_backward's grad_w length)
        alloc = _TORCH_ALLOCATOR if use_torch_allocator else None
        flags = (PR_BUILD_CSR if build_csr else 0) | (PR_DEDUP if dedup else 0)
        self.handle = pr_graph_create(n, src, dst, w, flags, alloc, stream)
        self.weighted = w is not None

    def close(self):
        if getattr(self, "handle", None):
            pr_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return pr_graph_info(self.handle)

    def export(self, csr=False, stream=None):
        return pr_graph_export(self.handle, stream, csr)

    def solve(self, out=None, stream=None, **kw):
        x = out if out is not None else torch.empty(self.n, dtype=torch.float64, device="cuda")
        res = pr_solve(self.handle, make_options(**kw), x, stream)
        return x, res

    def solve_batched(self, seeds=None, out=None, stream=None, V=None, **kw):
        kw.setdefault("precision", "fp32")
        B = int(seeds.numel()) if seeds is not None else int(V.shape[1])
        dt = torch.float64 if kw["precision"] == "fp64" else torch.float32
        X = out if out is not None else torch.empty((self.n, B), dtype=dt, device="cuda")
        res = pr_solve_batched(self.handle, make_options(**kw), seeds, X, stream, V=V)
        return X, res

    def backward(self, x, grad_x, stream=None, want_w=True, want_d=True, **kw):
        gw = torch.empty(self.m, dtype=torch.float64, device="cuda") if want_w else None
        gd = torch.empty(1, dtype=torch.float64, device="cuda") if want_d else None
        res = pr_backward(self.handle, make_options(**kw), x, grad_x, gw, gd, stream)
        return gw, gd, res


def solve_multi(graphs, outs=None, stream=None, **kw):
    """Solves several graphs together (pr_solve_multi); returns the result
    vectors (float64, input ids) and one PrResult per graph."""
    xs = outs if outs is not None else [torch.empty(g.n, dtype=torch.float64, device="cuda")
                                        for g in graphs]
    res = pr_solve_multi([g.handle for g in graphs], make_options(**kw), xs, stream)
    return xs, res


class PageRankFn(torch.autograd.Function):
    """x = PageRank of the graph (src -> dst, n vertices) with raw edge weights
    w (row-normalised inside) and damping d, differentiable in w and d.

    ``PageRankFn.apply(w, d, src, dst, n, opts)``: w float tensor [m] on the
    GPU, d a 0-dim tensor, src/dst int32 device tensors, opts a dict of solve
    options (threshold, max_iter, precision of the forward, ``adjoint`` =
    options of the reverse solve).  Backward returns (dL/dw, dL/dd, None, ...)
    from pr_backward's adjoint solve at the forward's fixed point."""

    @staticmethod
    def forward(ctx, w, d, src, dst, n, opts=None):
        opts = dict(opts or {})
        adj = dict(opts.pop("adjoint", {}))
        g = Graph(n, src, dst, w=w.detach().to(torch.float32).contiguous())
        x, _ = g.solve(d=float(d), **opts)
        ctx.graph, ctx.d, ctx.adj = g, float(d), adj
        ctx.w_dtype, ctx.d_dtype = w.dtype, d.dtype
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, grad_x):
        (x,) = ctx.saved_tensors
        g = ctx.graph
        adj = dict(ctx.adj)
        adj.setdefault("threshold", 1e-13)
        gw, gd, _ = g.backward(x, grad_x.to(torch.float64).contiguous(), d=ctx.d, **adj)
        g.close()
        ctx.graph = None
        return (gw.to(ctx.w_dtype), gd.reshape(()).to(ctx.d_dtype), None, None, None, None)
