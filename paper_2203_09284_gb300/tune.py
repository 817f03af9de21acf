"""Launch-parameter search: for a graph (or a family of graphs solved
together) time sweeps under each candidate `PrTune` on the device and keep
the fastest.  Results can be cached in a JSON file keyed by the device and
the graph's shape, so a later run with the same kind of graph skips the
search.  The sweep's work decomposition depends on these parameters only
for speed: every candidate computes the same iterates (summation order
aside), which the parity tests check."""
from __future__ import annotations

import json
import os
from itertools import product

# (t_lo, t_hub, hub_seg, tile, stage_kb, mid_wide)
DEFAULT_CANDIDATES = [
    dict(t_lo=t_lo, t_hub=t_hub, hub_seg=seg, tile=tile, stage_kb=stage, mid_wide=wide)
    for t_lo, (t_hub, seg), tile, stage, wide in product(
        (16, 32), ((1024, 2048), (4096, 4096)), (128, 256), (32, 64), (256, 1024))
]


def graph_signature(info: dict, device_name: str, precision: str, variant: str) -> str:
    """Cache key: device, sweep kind and the graph's vertex, edge and dangling
    counts rounded to two significant digits (graphs of one family share
    it; the class sizes are left out: they follow the last launch
    parameters used)."""
    def r2(v):
        v = int(v)
        if v < 100:
            return v
        s = len(str(v)) - 2
        return round(v, -s)
    return "|".join(str(x) for x in (device_name, precision, variant, r2(info["n"]),
                                      r2(info["m"]), r2(info["n_dangling"])))


def sweep_time_ms(solve, sweeps: int = 8, reps: int = 2) -> float:
    """Device time of one sweep: (time of 1 + sweeps sweeps - time of 1) /
    sweeps, each the best of `reps` runs timed with CUDA events."""
    import torch

    def run(k):
        best = None
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            solve(k)
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b)
            best = t if best is None or t < best else best
        return best

    return (run(1 + sweeps) - run(1)) / sweeps


def search(time_of, candidates=None):
    """The candidate with the smallest time_of(candidate) (ties: the first);
    returns (best, {index: time})."""
    cands = list(candidates or DEFAULT_CANDIDATES)
    times = {}
    best_i = None
    for i, c in enumerate(cands):
        t = float(time_of(c))
        times[i] = t
        if best_i is None or t < times[best_i]:
            best_i = i
    return cands[best_i], times


def _load_cache(path):
    if path and os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def _store_cache(path, cache):
    if not path:
        return
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune(graph, precision="fp32", variant="jacobi", candidates=None, sweeps=8, cache=None,
             x_out=None):
    """Best launch parameters (a dict for `tune=`) for sweeps of `graph`.

    graph      a paper_2203_09284_gb300.Graph
    precision  "fp64" or "fp32" (the sweep whose speed is searched; the
               defect-correction forms run the FP32 sweep)
    cache      path of a JSON cache, or None
    Returns (tune, report) with report = {"key", "cached", "times_ms"}.
    """
    import torch
    info = graph.info()
    key = graph_signature(info, torch.cuda.get_device_name(), precision, variant)
    store = _load_cache(cache)
    if key in store:
        return dict(store[key]["tune"]), {"key": key, "cached": True,
                                          "times_ms": store[key]["times_ms"]}
    x = x_out if x_out is not None else torch.empty(graph.n, dtype=torch.float64,
                                                    device="cuda")

    def time_of(c):
        return sweep_time_ms(lambda k: graph.solve(out=x, variant=variant, precision=precision,
                                                   threshold=0.0, max_iter=k, tune=c), sweeps)

    best, times = search(time_of, candidates)
    cands = list(candidates or DEFAULT_CANDIDATES)
    report = {str(i): round(t, 5) for i, t in times.items()}
    store[key] = {"tune": best, "times_ms": report, "candidates": cands}
    _store_cache(cache, store)
    return dict(best), {"key": key, "cached": False, "times_ms": report}


def autotune_multi(graphs, precision="fp32", candidates=None, sweeps=8):
    """Best launch parameters for solving `graphs` together (pr_solve_multi):
    each candidate is timed on the whole family's sweeps."""
    from . import solve_multi

    def time_of(c):
        return sweep_time_ms(lambda k: solve_multi(graphs, precision=precision, threshold=0.0,
                                                   max_iter=k, tune=c), sweeps)

    best, times = search(time_of, candidates)
    return dict(best), {str(i): round(t, 5) for i, t in times.items()}
