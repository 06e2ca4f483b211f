"""The decode server: continuous batching over mixed distances.

* A request decoded alone and the same request inside a concurrent mix of
  other requests (admitted while others run) give identical results, both
  equal to xzzx_decode_batch on that syndrome alone (shot index = request id).
* Every result of the mix equals its own decode_batch call; small-distance
  results equal the oracle.
* Counters and latency percentiles are consistent; a full queue rejects.
"""
import time

import numpy as np
import pytest

import oracle as O
from layout import syn_bits_to_words, words_to_labels

pytestmark = pytest.mark.gpu

SEED, R, N, B0, B1 = 0x5E77E, 8, 120, 0.05, 20.0
CLASSES = [(3, 0.10, 10), (5, 0.15, 100), (9, 0.15, 100), (17, 0.12, 100), (21, 0.10, 10)]


@pytest.fixture(scope="module")
def env():
    from paper_2509_17837_gb300 import build
    build.build()
    import torch

    import paper_2509_17837_gb300 as X
    return X, torch


def make_server(X, **kw):
    # batches of at most 4 requests anneal one warp per chain, larger ones one
    # thread per chain: the probe below runs alone in the first mode and in
    # the mix mostly in the second
    sv = X.Server(SEED, R, N, B0, B1, max_batch=kw.get("max_batch", 16), n_slots=kw.get("n_slots", 3),
                  queue_capacity=kw.get("queue_capacity", 100000), warp_max_requests=4)
    ids = []
    for d, p, eta in CLASSES:
        ids.append(sv.add_class(d, X.noise_from_eta(p, eta)))
    sv.start()
    return sv, ids


def syndromes_for(d, p, eta, n, seed):
    pxyz = O.noise_from_eta(p, eta)
    err, syn = O.sample(d, pxyz, seed, 0, n)
    w = syn_bits_to_words(syn)
    out = np.zeros((n, 32), np.uint32)
    out[:, :w.shape[1]] = w
    return err, syn, out


def wait_for(sv, n, timeout_s=60.0):
    res, t0 = [], time.time()
    while len(res) < n and time.time() - t0 < timeout_s:
        res += sv.poll(timeout_ms=200)
    assert len(res) == n, (len(res), n)
    return res


def reference(X, torch, d, p, eta, syn_words, req_id):
    code = X.Code(d)
    noise = X.noise_from_eta(p, eta)
    sched = X.Schedule(noise, N, B0, B1)
    sw = code.syn_words
    syn = torch.from_numpy(syn_words[None, :sw].astype(np.uint32).view(np.int32)).cuda()
    out = X.decode_batch(code, noise, sched, SEED, req_id, syn, R)
    torch.cuda.synchronize()
    return int(out["cls"][0]), out["E4"][0].cpu().tolist(), out["recovery"][0].cpu().numpy().view(np.uint32).tolist()


def test_alone_equals_in_the_mix(env):
    X, torch = env
    sv, cids = make_server(X)
    try:
        # alone
        d, p, eta = CLASSES[2]
        _, _, syn = syndromes_for(d, p, eta, 1, 7)
        assert sv.submit(1000, cids[2], syn[0]) == 0
        alone = wait_for(sv, 1)[0]
        # in the mix: 150 requests of all classes arriving over ~20 ms, the
        # probe among them, admitted while earlier batches run
        rng = np.random.default_rng(3)
        ids, cls, syns, meta = [], [], [], {}
        for k in range(150):
            c = int(rng.integers(0, len(CLASSES)))
            dd, pp, ee = CLASSES[c]
            _, _, s = syndromes_for(dd, pp, ee, 1, 100 + k)
            ids.append(2000 + k)
            cls.append(cids[c])
            syns.append(s[0])
            meta[2000 + k] = (c, s[0])
        ids.insert(75, 1000)
        cls.insert(75, cids[2])
        syns.insert(75, syn[0])
        arrivals = np.sort(rng.uniform(0, 20000, len(ids)))
        sv.replay(ids, cls, np.stack(syns), arrivals)
        mix = {r["req_id"]: r for r in wait_for(sv, len(ids))}
        probe = mix[1000]
        assert (probe["cls"], probe["E4"], probe["recovery"]) == (alone["cls"], alone["E4"], alone["recovery"])
        assert (alone["cls"], alone["E4"], alone["recovery"]) == reference(X, torch, d, p, eta, syn[0], 1000)
        st = sv.stats()
        assert st["completed"] == len(ids) + 1 and st["rejected"] == 0
        assert st["batches"] >= 3 and st["p99_us"] >= st["p50_us"] > 0
        # every request of the mix equals its own decode_batch call
        for rid, (c, s) in list(meta.items())[::5]:
            dd, pp, ee = CLASSES[c]
            r = mix[rid]
            assert (r["cls"], r["E4"], r["recovery"]) == reference(X, torch, dd, pp, ee, s, rid), rid
        # and small distances equal the oracle
        for rid, (c, s) in meta.items():
            dd, pp, ee = CLASSES[c]
            if dd > 5:
                continue
            pxyz = O.noise_from_eta(pp, ee)
            from layout import syn_words_to_bits
            bits = syn_words_to_bits(s[None, :(dd * dd - 1 + 31) // 32], dd * dd - 1)
            ref = O.decode(dd, pxyz, 1024, O.LINEAR, N, B0, B1, SEED, rid, R, bits)
            r = mix[rid]
            assert r["cls"] == ref["cls"][0] and r["E4"] == list(ref["E4"][0])
            w = (dd * dd + 31) // 32
            assert np.array_equal(words_to_labels(np.array(r["recovery"], np.uint32)[None], dd * dd)[0],
                                  ref["recovery"][0])
    finally:
        sv.close()


def test_full_queue_rejects(env):
    X, torch = env
    sv, cids = make_server(X, queue_capacity=4, n_slots=1, max_batch=1)
    try:
        d, p, eta = CLASSES[4]
        _, _, syn = syndromes_for(d, p, eta, 40, 9)
        codes = [sv.submit(5000 + k, cids[4], syn[k]) for k in range(40)]
        from paper_2509_17837_gb300._lib import XZZX_EBUSY
        assert XZZX_EBUSY in codes
        accepted = sum(c == 0 for c in codes)
        res = wait_for(sv, accepted)
        st = sv.stats()
        assert st["rejected"] == codes.count(XZZX_EBUSY) and st["completed"] == accepted == len(res)
    finally:
        sv.close()


def test_slot_too_small_for_one_request_is_refused(env):
    """A budget whose slots cannot hold one request of a registered class is
    refused at start (XZZX_ENOMEM) instead of leaving that class's requests
    waiting forever; closing the refused server returns."""
    X, torch = env
    from paper_2509_17837_gb300._lib import XZZX_ENOMEM
    sv = X.Server(SEED, 64, N, B0, B1, max_batch=16, n_slots=8, hbm_budget_bytes=64 << 10)
    try:
        sv.add_class(21, X.noise_from_eta(0.1, 10))
        with pytest.raises(X.XzzxError) as e:
            sv.start()
        assert e.value.status == XZZX_ENOMEM
    finally:
        sv.close()
