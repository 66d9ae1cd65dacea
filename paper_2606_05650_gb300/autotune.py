"""Autotuner of the codec's launch shapes.

The tunables (gsnfs_tune_set: RAHT tile size, CTAs per SM of the first
transform pass and of the prelude tile passes, pipelined or plain first
transform pass) change how the work is tiled
and spread over the 152 SMs, never what is computed, so the tuner may pick
any of them: it checks on every candidate that the bitstreams and the decoded
frames are byte-identical to the default's and drops a candidate that is not.

Search: coordinate descent over the tunables in a fixed order, each swept
over its candidate list with the others held at their best so far; a
candidate must beat the best time by 1% to be taken.  Results are cached in a
JSON file (GSNFS_TUNE_CACHE, else ~/.cache/gsnfs/tune.json) keyed by device
name, channel count, frame-size bucket (nearest power of two) and frames per
call.
"""
from __future__ import annotations

import json
import math
import os

ORDER = ("raht_pipe", "raht_tile", "raht_grid", "prelude_grid")
CANDIDATES = {"raht_pipe": [0, 1, 2], "raht_tile": [0, 512, 1024], "raht_grid": [0, 2, 3, 6, 8], "prelude_grid": [0, 4, 16]}


def default_cache_path() -> str:
    return os.environ.get("GSNFS_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "gsnfs", "tune.json"))


def workload_key(device_name: str, C: int, n_per_frame: int, frames: int) -> str:
    bucket = 1 << max(0, round(math.log2(max(n_per_frame, 1))))
    return f"{device_name}|C={C}|n~{bucket}|F={frames}"


def coordinate_descent(measure, order=ORDER, candidates=None, gain=0.01, same=lambda a, b: a == b):
    """measure(params) -> (ms, outputs) or None when the setting cannot run.
    Returns (best params, best ms, default ms, trials).  A candidate whose
    outputs differ from the default's (same(ref, outputs) false) is rejected."""
    candidates = candidates or CANDIDATES
    best = {k: 0 for k in order}
    r = measure(dict(best))
    if r is None:
        raise RuntimeError("the default launch shapes do not run")
    default_ms, ref_sig = r
    best_ms = default_ms
    trials = [(dict(best), default_ms, True)]
    for name in order:
        for v in candidates[name]:
            if v == best[name]:
                continue
            p = dict(best)
            p[name] = v
            r = measure(p)
            if r is None:
                trials.append((p, None, False))
                continue
            ms, sig = r
            ok = bool(same(ref_sig, sig))
            del sig
            trials.append((p, ms, ok))
            if ok and ms < best_ms * (1.0 - gain):
                best, best_ms = p, ms
    return best, best_ms, default_ms, trials


def load(key: str, path: str | None = None):
    path = path or default_cache_path()
    try:
        with open(path) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def save(key: str, entry: dict, path: str | None = None):
    path = path or default_cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[key] = entry
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(params: dict, device=None):
    from . import gsnfs as G
    for name in ORDER:
        G.tune_set(name, int(params.get(name, 0)), device)


def tune_round_trip(pos_list, attr_list, J_list, qp, reps: int = 3, cache: str | None = None, use_cache=True):
    """Tunes the batched encode + decode of these frames on their device and
    leaves the best setting applied.  Returns the cache entry."""
    import torch
    from . import gsnfs as G
    dev = pos_list[0].device
    F = len(pos_list)
    n = max(int(p.shape[0]) for p in pos_list)
    key = workload_key(torch.cuda.get_device_name(dev), qp.C, n, F)
    if use_cache:
        hit = load(key, cache)
        if hit:
            apply(hit["params"], dev)
            return dict(hit, cached=True)
    stream = torch.cuda.current_stream(dev)
    rows_cap = sum(int(p.shape[0]) for p in pos_list)
    state = {"out": None}

    def run():
        out, offs = G.encode_batch(pos_list, attr_list, J_list, [1.0], qp, out=state["out"])
        state["out"] = out
        pos, attr, rows = G.decode_batch(out, offs, qp.C, rows_cap)
        return out, offs, pos, attr

    def measure(params):
        try:
            apply(params, dev)
            run()  # carve / warm
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                out, offs, pos, attr = run()
            e1.record(stream)
            torch.cuda.synchronize()
        except G.GsnfsError:
            return None
        n_out = int(offs[-1])
        # the outputs themselves (device copies), compared byte for byte
        return e0.elapsed_time(e1) / reps, (out[:n_out].clone(), pos.clone(), None if attr is None else attr.clone())

    def same(a, b):
        return all((x is None and y is None) or (x is not None and y is not None and x.shape == y.shape
                                                  and torch.equal(x, y)) for x, y in zip(a, b))

    best, best_ms, default_ms, trials = coordinate_descent(measure, same=same)
    apply(best, dev)
    entry = {"params": best, "ms": round(best_ms, 4), "default_ms": round(default_ms, 4),
             "trials": [[p, None if m is None else round(m, 4), ok] for p, m, ok in trials]}
    if use_cache:
        save(key, entry, cache)
    return dict(entry, cached=False, key=key)
