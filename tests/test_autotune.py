"""Autotuner search and cache (host logic, no GPU): coordinate descent finds
the fastest admissible setting, rejects settings whose outputs differ from
the default's or that cannot run, and the JSON cache round-trips."""
from paper_2606_05650_gb300 import autotune as at


def _fake(times, wrong=(), broken=()):
    calls = []

    def measure(p):
        key = tuple(p[k] for k in at.ORDER)
        calls.append(key)
        if key in broken:
            return None
        return times(p), ("bad" if key in wrong else "ref")
    return measure, calls


def test_descent_finds_the_separable_optimum():
    cost = {"raht_pipe": {0: 1, 1: 2, 2: 1.5}, "raht_tile": {0: 5, 512: 3, 1024: 4},
            "raht_grid": {0: 5, 2: 6, 3: 4, 6: 2, 8: 3}, "prelude_grid": {0: 1, 4: 2, 16: 0.5}}
    measure, calls = _fake(lambda p: sum(cost[k][p[k]] for k in at.ORDER))
    best, ms, d, trials = at.coordinate_descent(measure)
    assert best == {"raht_pipe": 0, "raht_tile": 512, "raht_grid": 6, "prelude_grid": 16}
    assert ms == 1 + 3 + 2 + 0.5 and d == 12
    assert len(calls) == 1 + 2 + 2 + 4 + 2  # default, then each other candidate once


def test_descent_rejects_wrong_outputs_broken_runs_and_small_gains():
    def t(p):
        return {0: 10.0, 512: 5.0, 1024: 9.95}[p["raht_tile"]] + {0: 0, 2: -1, 3: 0, 6: 0, 8: 0}[p["raht_grid"]]
    measure, _ = _fake(t, wrong={(0, 512, 0, 0)}, broken={(0, 0, 2, 0)})
    best, ms, d, trials = at.coordinate_descent(measure)
    # pipe off no faster, tile 512 wrong, 1024 < 1% gain, grid 2 broken
    assert best == {"raht_pipe": 0, "raht_tile": 0, "raht_grid": 0, "prelude_grid": 0}
    assert ms == d == 10.0
    assert any(p["raht_tile"] == 512 and ok is False for p, m, ok in trials)
    assert any(p["raht_grid"] == 2 and m is None for p, m, ok in trials)


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    k1 = at.workload_key("GB300", 56, 1_000_000, 8)
    k2 = at.workload_key("GB300", 56, 1_100_000, 8)
    assert k1 == k2 and k1 != at.workload_key("GB300", 3, 1_000_000, 8)
    assert at.load(k1, path) is None
    at.save(k1, {"params": {"raht_tile": 512}, "ms": 1.0}, path)
    at.save("other", {"params": {}}, path)
    assert at.load(k1, path)["params"] == {"raht_tile": 512}
