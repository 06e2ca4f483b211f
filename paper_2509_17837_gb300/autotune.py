"""Autotuner for batched decoding.

It picks, for a batch shape, by timing short runs:

* the chain-to-hardware mapping, as the launch mode of ``Batch.run``:
  0 = one persistent launch, one chain per thread, CTAs pulling chunks of
  chains from a queue; 1 = one launch per distance, one chain per thread;
  2 = one launch per distance, one chain per warp; 3 = each distance's own
  launch, concurrently on forked streams; 4 = one persistent launch per
  distance class, concurrently on forked streams;
* for mode 0, the persistent grid in CTAs per SM (how many chains are in
  flight per SM; 0 = the occupancy limit) and the order of the chunk queue
  (0 = longest chunks first, 1 = segment order);
* the chains per CTA of the annealing launches (128 or 256: the chunk size,
  one CTA per chunk) and the unroll of the kernels' sweep loop (1 or 2), each
  a separately compiled kernel variant.

The choice is cached in a JSON file keyed by GPU name and batch shape.  The
knobs only change scheduling and code shape: every choice decodes
bit-identically.
"""
import json
import os
import time

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")
KEY_VERSION = "v3"

# (mode, ctas_per_sm, order, chains_per_cta, sweep_unroll)
DEFAULT_CANDIDATES = ([(0, c, o, nt, 1) for c in (0, 2, 4) for o in (0, 1) for nt in (128, 256)] +
                      [(0, 0, 0, nt, 2) for nt in (128, 256)] +
                      [(m, 0, 0, nt, u) for m in (1, 3) for nt in (128, 256) for u in (1, 2)] + [(2, 0, 0, 128, 1)] +
                      [(4, c, 0, nt, 1) for c in (0, 2) for nt in (128, 256)])


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, cache):
    tmp = path + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def shape_key(segments, device_name):
    """Batch shape: distances, restarts, sweeps and shot counts (not the data)."""
    parts = sorted((sg["code"].d, sg["restarts"], sg["sched"].n_sweeps) for sg in segments)
    shots = sum(int(sg["syndromes"].shape[0]) for sg in segments)
    dist = {}
    for d, r, n in parts:
        dist[(d, r, n)] = dist.get((d, r, n), 0) + 1
    return "%s|%s|%s|shots=%d" % (KEY_VERSION, device_name, sorted(dist.items()), shots)


_CURRENT = object()


def tune(make_batch, segments, candidates=None, reps=1, use_cache=True, cache_path=None, device_name=None,
         stream=_CURRENT, sync=None):
    """Time each candidate (mode, ctas_per_sm, order, chains_per_cta,
    sweep_unroll) and return (best, timings).

    make_batch(ctas_per_sm, order, chains_per_cta, sweep_unroll) -> an object
    with run(mode, stream) and close().  stream / sync default to the current
    CUDA stream and torch.cuda.synchronize; device_name to the current GPU's
    name.
    """
    if device_name is None or stream is _CURRENT or sync is None:
        import torch
        device_name = device_name or torch.cuda.get_device_name()
        stream = torch.cuda.current_stream() if stream is _CURRENT else stream
        sync = sync or torch.cuda.synchronize
    path = cache_path or CACHE
    key = shape_key(segments, device_name)
    cache = _load(path) if use_cache else {}
    if use_cache and key in cache:
        return tuple(cache[key]["cfg"]), cache[key].get("timings", {})
    timings = {}
    for cand in (candidates or DEFAULT_CANDIDATES):
        mode, cps, order, nt, unroll = cand
        b = make_batch(cps, order, nt, unroll)
        try:
            b.run(mode, stream)  # warm-up
            sync()
            best_s = float("inf")
            for _ in range(reps):  # the fastest of reps runs: robust to one-off interference
                t0 = time.perf_counter()
                b.run(mode, stream)
                sync()
                best_s = min(best_s, time.perf_counter() - t0)
            timings[",".join(str(x) for x in cand)] = best_s
        finally:
            b.close()
    best = min(timings, key=timings.get)
    cfg = tuple(int(x) for x in best.split(","))
    if use_cache:
        cache[key] = {"cfg": list(cfg), "timings": timings}
        _save(path, cache)
    return cfg, timings
