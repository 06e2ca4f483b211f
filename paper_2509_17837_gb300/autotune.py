"""Autotuner for batched decoding: picks the persistent grid (CTAs per SM) and
the chunk-queue order for a batch shape by timing short runs, and caches the
choice in a JSON file keyed by GPU name and batch shape.

The knobs only change scheduling: every choice decodes bit-identically.
"""
import json
import os
import time

import torch

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(cache):
    tmp = CACHE + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def shape_key(segments):
    """Batch shape: distances, restarts, sweeps and shot counts (not the data)."""
    parts = sorted((sg["code"].d, sg["restarts"], sg["sched"].n_sweeps) for sg in segments)
    shots = sum(int(sg["syndromes"].shape[0]) for sg in segments)
    dist = {}
    for d, r, n in parts:
        dist[(d, r, n)] = dist.get((d, r, n), 0) + 1
    return "%s|%s|shots=%d" % (torch.cuda.get_device_name(), sorted(dist.items()), shots)


def tune(make_batch, segments, candidates=None, reps=1, use_cache=True):
    """make_batch(ctas_per_sm, order) -> Batch.  Returns (best_cfg, timings)."""
    key = shape_key(segments)
    cache = _load() if use_cache else {}
    if use_cache and key in cache:
        return tuple(cache[key]["cfg"]), cache[key].get("timings", {})
    if candidates is None:
        candidates = [(c, o) for c in (0, 1, 2, 3, 4) for o in (0, 1)]
    timings = {}
    stream = torch.cuda.current_stream()
    for cps, order in candidates:
        b = make_batch(cps, order)
        b.run(0, stream)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            b.run(0, stream)
        torch.cuda.synchronize()
        timings["%d,%d" % (cps, order)] = (time.perf_counter() - t0) / reps
        b.close()
    best = min(timings, key=timings.get)
    cfg = tuple(int(x) for x in best.split(","))
    if use_cache:
        cache[key] = {"cfg": list(cfg), "timings": timings}
        _save(cache)
    return cfg, timings
