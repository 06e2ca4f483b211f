"""CPU checks of the batch autotuner's logic with a fake batch: it times every
candidate, picks the fastest (mode, ctas_per_sm, order, chains_per_cta,
sweep_unroll), caches the choice by GPU and batch shape, and serves a
repeated shape from the cache without timing again."""
import time
from types import SimpleNamespace

from paper_2509_17837_gb300 import autotune


class FakeBatch:
    def __init__(self, cps, order, nt, unroll, log, cost):
        self.knobs, self.log, self.cost = (cps, order, nt, unroll), log, cost

    def run(self, mode, stream):
        self.log.append((mode,) + self.knobs)
        time.sleep(self.cost((mode,) + self.knobs))

    def close(self):
        pass


def segments(shots):
    seg = lambda d, r, n, s: dict(code=SimpleNamespace(d=d), restarts=r, sched=SimpleNamespace(n_sweeps=n),
                                  syndromes=SimpleNamespace(shape=(s, 4)))
    return [seg(5, 16, 500, shots), seg(21, 64, 2000, shots)]


def test_picks_fastest_and_caches(tmp_path):
    log = []
    fastest = (1, 0, 0, 256, 2)
    assert fastest in autotune.DEFAULT_CANDIDATES
    cost = lambda cand: 0.002 if cand == fastest else 0.004
    make = lambda cps, order, nt, unroll: FakeBatch(cps, order, nt, unroll, log, cost)
    kw = dict(cache_path=str(tmp_path / "cache.json"), device_name="fake-gpu", stream=None, sync=lambda: None)
    cfg, timings = autotune.tune(make, segments(100), **kw)
    assert cfg == fastest
    assert set(timings) == {",".join(str(x) for x in c) for c in autotune.DEFAULT_CANDIDATES}
    assert {c for c in log} == set(autotune.DEFAULT_CANDIDATES)       # every candidate ran
    n = len(log)
    cfg2, _ = autotune.tune(make, segments(100), **kw)                  # same shape: from the cache
    assert cfg2 == cfg and len(log) == n
    cfg3, _ = autotune.tune(make, segments(200), **kw)                  # another shape: timed again
    assert cfg3 == cfg and len(log) > n


def test_shape_key_ignores_data_but_not_shape():
    a = autotune.shape_key(segments(100), "g")
    assert a == autotune.shape_key(list(reversed(segments(100))), "g")
    assert a != autotune.shape_key(segments(101), "g")
    assert a != autotune.shape_key(segments(100), "h")
