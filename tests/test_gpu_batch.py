"""Uneven batches: many segments with different distances, noise classes,
schedules and restart counts in one run.  The persistent launch (mode 0), the
one-launch-per-distance form (mode 1) and graph replays must all equal
xzzx_decode_batch on each segment alone, bit for bit, and every segment must
equal the oracle."""
import numpy as np
import pytest

import oracle as O
from layout import words_to_labels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2509_17837_gb300 import build
    build.build()
    import torch

    import paper_2509_17837_gb300 as X
    return X, torch


SEG_SPECS = [  # d, p, eta, restarts, sweeps, n_shots, shot0
    (3, 0.10, 10, 4, 40, 33, 0),
    (5, 0.12, 1, 4, 50, 20, 1000),
    (7, 0.18, 100, 8, 60, 9, 7),
    (9, 0.20, 10, 8, 80, 5, 11),
    (13, 0.15, 100, 8, 40, 3, 500),
    (5, 0.08, 100, 6, 30, 17, 99),
    (17, 0.15, 100, 4, 30, 2, 3),
    (21, 0.12, 10, 4, 20, 2, 0),
]


def make_segments(X, torch, seed, with_errors=True):
    segs = []
    for d, p, eta, R, N, n, shot0 in SEG_SPECS:
        code = X.Code(d)
        noise = X.noise_from_eta(p, eta)
        sched = X.Schedule(noise, N, 0.05, 20.0)
        err, syn = X.sample_errors(code, noise, seed, shot0, n)
        segs.append(dict(code=code, noise=noise, sched=sched, shot0=shot0, syndromes=syn, restarts=R,
                         true_errors=err if with_errors else None))
    return segs


def reference_outputs(X, torch, segs, seed):
    refs = []
    for sg in segs:
        refs.append(X.decode_batch(sg["code"], sg["noise"], sg["sched"], seed, sg["shot0"], sg["syndromes"],
                                   sg["restarts"], true_errors=sg["true_errors"]))
    torch.cuda.synchronize()
    return refs


def assert_same(outs, refs):
    for j, (o, r) in enumerate(zip(outs, refs)):
        for k in ("cls", "E4", "recovery", "fail"):
            if r.get(k) is None:
                continue
            assert np.array_equal(o[k].cpu().numpy(), r[k].cpu().numpy()), (j, k)


def test_batch_modes_match_per_segment_calls(env):
    X, torch = env
    seed = 0xB47C
    segs = make_segments(X, torch, seed)
    refs = reference_outputs(X, torch, segs, seed)
    b = X.Batch(segs, seed)
    info = b.info()
    assert info["n_segments"] == len(SEG_SPECS) and info["n_distances"] == 7
    assert info["launches_batched"] == 4 and info["launches_plain"] == 21  # greedy with and without lists
    for mode in (0, 1, 2, 3, 4, 0, 3, 4):   # second runs reuse the reset queues and the side streams
        for o in b.outputs:
            for t in o.values():
                if t is not None:
                    t.fill_(0x5A)
        b.run(mode)
        torch.cuda.synchronize()
        assert_same(b.outputs, refs)
    s = torch.cuda.Stream()
    for _ in range(2):                # capture, then replay
        for o in b.outputs:
            o["cls"].fill_(7)
        with torch.cuda.stream(s):
            b.run_graph(s)
        s.synchronize()
        assert_same(b.outputs, refs)


@pytest.mark.parametrize("graph_mode", [3, 4])
def test_batch_concurrent_mode_graph(env, graph_mode):
    """Modes 3 (each distance's own launch on forked streams) and 4 (one
    persistent launch per distance class on forked streams) captured as a
    CUDA graph and replayed: identical outputs to the per-segment calls."""
    X, torch = env
    seed = 0x3C0C
    segs = make_segments(X, torch, seed)
    refs = reference_outputs(X, torch, segs, seed)
    b = X.Batch(segs, seed, graph_mode=graph_mode)
    assert b.info()["n_classes"] == 2
    s = torch.cuda.Stream()
    for _ in range(3):
        for o in b.outputs:
            for t in o.values():
                if t is not None:
                    t.fill_(0x3C)
        with torch.cuda.stream(s):
            b.run_graph(s)
        s.synchronize()
        assert_same(b.outputs, refs)
    with pytest.raises(X.XzzxError):
        X.Batch(segs, seed, graph_mode=1)


def test_batch_segments_match_oracle(env):
    """Every segment of the batch, d = 3 to 21, equals the oracle's decode."""
    X, torch = env
    seed = 0x0AC1E
    segs = make_segments(X, torch, seed)
    b = X.Batch(segs, seed, ctas_per_sm=1, order=1)
    b.run(0)
    torch.cuda.synchronize()
    for sg, o, spec in zip(segs, b.outputs, SEG_SPECS):
        d, p, eta, R, N, n, shot0 = spec
        noise = sg["noise"]
        pxyz = (noise.px, noise.py, noise.pz)
        oerr, osyn = O.sample(d, pxyz, seed, shot0, n)
        ref = O.decode(d, pxyz, noise.scale, O.LINEAR, N, 0.05, 20.0, seed, shot0, R, osyn, oerr)
        assert np.array_equal(o["cls"].cpu().numpy(), ref["cls"])
        assert np.array_equal(o["E4"].cpu().numpy(), ref["E4"])
        assert np.array_equal(words_to_labels(o["recovery"].cpu().numpy(), d * d), ref["recovery"])
        assert np.array_equal(o["fail"].cpu().numpy(), ref["fail"])


def test_batch_rejects_bad_segments(env):
    X, torch = env
    from paper_2509_17837_gb300._lib import XzzxError
    segs = make_segments(X, torch, 1)[:2]
    segs[1]["restarts"] = 0
    with pytest.raises(XzzxError):
        X.Batch(segs, 1)


@pytest.mark.parametrize("nt,unroll", [(128, 1), (128, 2), (256, 1), (256, 2)])
def test_batch_tuning_variants_identical(env, nt, unroll):
    """Every (chains per CTA, sweep unroll) variant of the batched annealing
    kernels decodes bit-identically to per-segment xzzx_decode_batch, in the
    persistent, per-distance and concurrent forms."""
    X, torch = env
    seed = 0x7A11
    segs = make_segments(X, torch, seed)
    refs = reference_outputs(X, torch, segs, seed)
    b = X.Batch(segs, seed, chains_per_cta=nt, sweep_unroll=unroll)
    info = b.info()
    assert info["chains_per_cta"] == nt and info["sweep_unroll"] == unroll
    for mode in (0, 1, 3, 4):
        for o in b.outputs:
            o["cls"].fill_(9)
        b.run(mode)
        torch.cuda.synchronize()
        assert_same(b.outputs, refs)
    with pytest.raises(X.XzzxError):
        X.Batch(segs, seed, chains_per_cta=64)


@pytest.mark.parametrize("cap", [1, 2, 4])
def test_batch_warp_mapping_occupancy_cap(env, cap):
    """Mode 2 (one warp per chain) with its resident CTAs per SM capped by
    padded shared memory: at most cap CTAs per SM, and outputs identical to
    the per-segment calls."""
    X, torch = env
    seed = 0x3A9C
    segs = make_segments(X, torch, seed)
    refs = reference_outputs(X, torch, segs, seed)
    free = X.Batch(segs, seed)
    b = X.Batch(segs, seed, ctas_per_sm=cap)
    assert 1 <= b.info()["warp_ctas_per_sm"] <= cap
    assert free.info()["warp_ctas_per_sm"] >= b.info()["warp_ctas_per_sm"]
    b.run(2)
    torch.cuda.synchronize()
    assert_same(b.outputs, refs)
    free.close()
    b.close()


def test_batch_restarts_per_warp_match_per_segment_calls(env):
    """A batch large enough that its greedy launch gives each warp four
    restarts (segments d <= 15) decodes exactly as per-segment calls, whose
    own launches take two or one restarts per warp."""
    X, torch = env
    seed = 0x4E57
    specs = [(5, 0.12, 10, 16, 3000), (11, 0.16, 100, 64, 500), (17, 0.15, 100, 8, 200)]
    segs = []
    for d, p, eta, R, n in specs:
        code = X.Code(d)
        noise = X.noise_from_eta(p, eta)
        sched = X.Schedule(noise, 12, 0.05, 20.0)
        err, syn = X.sample_errors(code, noise, seed, 0, n)
        segs.append(dict(code=code, noise=noise, sched=sched, shot0=0, syndromes=syn, restarts=R, true_errors=err))
    refs = reference_outputs(X, torch, segs, seed)
    b = X.Batch(segs, seed)
    for mode in (0, 1):
        b.run(mode)
        torch.cuda.synchronize()
        assert_same(b.outputs, refs)
    b.close()
