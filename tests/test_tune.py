"""Host logic of the launch-parameter search (no GPU)."""
import json

from paper_2203_09284_gb300 import tune


def test_search_picks_the_fastest_first_on_ties():
    cands = [dict(tile=128), dict(tile=256), dict(tile=512), dict(tile=64)]
    times = {128: 3.0, 256: 1.5, 512: 1.5, 64: 2.0}
    best, got = tune.search(lambda c: times[c["tile"]], cands)
    assert best == dict(tile=256)
    assert got == {0: 3.0, 1: 1.5, 2: 1.5, 3: 2.0}


def test_default_candidates_are_distinct_and_complete():
    keys = {tuple(sorted(c.items())) for c in tune.DEFAULT_CANDIDATES}
    assert len(keys) == len(tune.DEFAULT_CANDIDATES) == 32
    assert all(set(c) == {"t_lo", "t_hub", "hub_seg", "tile", "stage_kb", "mid_wide"}
               for c in tune.DEFAULT_CANDIDATES)


def sa_eq(x, y):
    return (tune.graph_signature(x, "GB300", "fp32", "jacobi")
            == tune.graph_signature(y, "GB300", "fp32", "jacobi"))


def test_signature_groups_graphs_of_one_family():
    a = {"n": 4194304, "m": 67008246, "n_dangling": 419430, "bins": [3914232, 278278, 1794]}
    b = {"n": 4194304, "m": 67011000, "n_dangling": 419431, "bins": [3914000, 278100, 1790]}
    c = dict(a, m=33000000)
    assert sa_eq(a, dict(a, bins=[1, 2, 3]))
    sa = tune.graph_signature(a, "GB300", "fp32", "jacobi")
    assert sa == tune.graph_signature(b, "GB300", "fp32", "jacobi")
    assert sa != tune.graph_signature(c, "GB300", "fp32", "jacobi")
    assert sa != tune.graph_signature(a, "GB300", "fp64", "jacobi")


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert tune._load_cache(path) == {}
    tune._store_cache(path, {"k": {"tune": {"tile": 128}, "times_ms": {"0": 1.0}}})
    assert tune._load_cache(path)["k"]["tune"] == {"tile": 128}
    with open(path, "w") as f:
        f.write("{not json")
    assert tune._load_cache(path) == {}
    json.dumps(tune.DEFAULT_CANDIDATES)  # candidates are plain JSON
