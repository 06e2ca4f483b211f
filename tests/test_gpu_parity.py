"""GPU parity: every step of the CUDA path, called through the C ABI, against
the oracle on the same seeded inputs.  Everything is integer (or decided by an
integer comparison against a host FP64 table), so the bar is bit-exact:
errors, syndromes, greedy references and class bits, per-chain minimum
energies and configurations, decoded classes, coset energies, recoveries and
failure flags.
"""
import numpy as np
import pytest

import oracle as O
from layout import labels_to_words, syn_bits_to_words, syn_words_to_bits, words_to_labels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    from paper_2509_17837_gb300 import build
    build.build()
    import paper_2509_17837_gb300 as X
    return X


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def to_np(t):
    return t.cpu().numpy()


def gpu_words(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr).view(np.int32)).cuda()


@pytest.mark.parametrize("d,p,eta,conv", [(3, 0.1, 10, 0), (5, 0.2, 1.0, 1), (11, 0.16, 100, 0),
                                          (17, 0.3, 3, 0), (31, 0.25, 1000, 0)])
def test_sample_parity(X, torch, d, p, eta, conv):
    code = X.Code(d)
    noise = X.noise_from_eta(p, eta, conv)
    shot0, n = (1 << 33) + 5, 503                       # 64-bit shot index, ragged warp tail
    err, syn = X.sample_errors(code, noise, 0xABC, shot0, n)
    torch.cuda.synchronize()
    oe, osyn = O.sample(d, (noise.px, noise.py, noise.pz), 0xABC, shot0, n)
    assert np.array_equal(words_to_labels(to_np(err), d * d), oe)
    assert np.array_equal(syn_words_to_bits(to_np(syn), d * d - 1), osyn)


def oracle_noise(noise):
    return (noise.px, noise.py, noise.pz)


@pytest.mark.parametrize("d,p,eta,n,R", [(3, 0.1, 10, 64, 8), (5, 0.2, 3, 40, 6), (11, 0.22, 100, 30, 9),
                                         (17, 0.18, 100, 8, 5), (21, 0.2, 100, 6, 5), (31, 0.3, 1000, 3, 4)])
@pytest.mark.parametrize("randomised", [1, 0, 2])   # Alg. 6, Alg. 5, boundary initializer
def test_greedy_parity(X, torch, d, p, eta, n, R, randomised):
    code = X.Code(d)
    noise = X.noise_from_eta(p, eta)
    pxyz = oracle_noise(noise)
    _, osyn = O.sample(d, pxyz, 17, 100, n)
    syn = gpu_words(torch, syn_bits_to_words(osyn))
    init, cbits = X.greedy_init(code, noise, 17, 100, syn, R, randomised=randomised)
    torch.cuda.synchronize()
    init, cbits = to_np(init), to_np(cbits)
    LX, LZ = O.logicals(d)
    for s in range(n):
        for i in range(R):
            ref, _ = O.greedy(d, pxyz, noise.scale, 17, 100 + s, i, randomised, osyn[s])
            got = words_to_labels(init[s, i], d * d)
            assert np.array_equal(got, ref), (s, i)
            assert cbits[s, i] == O.class_bits(d, ref)  # class bits of R_i itself


@pytest.mark.parametrize("d,density", [(11, 0.5), (13, 0.9), (31, 0.3)])
def test_greedy_parity_dense_random_syndromes(X, torch, d, density):
    from inputs import random_syndromes
    code = X.Code(d)
    noise = X.make_noise(0.03, 0.05, 0.09)       # Wt_x != Wt_z: unequal matching weights
    pxyz = oracle_noise(noise)
    osyn = random_syndromes(d * d - 1, 4, density, seed=d)
    syn = gpu_words(torch, syn_bits_to_words(osyn))
    init, cbits = X.greedy_init(code, noise, 5, 7, syn, 3)
    torch.cuda.synchronize()
    init = to_np(init)
    for s in range(4):
        for i in range(3):
            ref, _ = O.greedy(d, pxyz, noise.scale, 5, 7 + s, i, 1, osyn[s])
            assert np.array_equal(words_to_labels(init[s, i], d * d), ref)


def anneal_case(X, torch, d, p, eta, n, R, kind, N, b0, b1, seed=3, shot0=11, scale=1024, per_warp=False,
                order=0, emin=0):
    code = X.Code(d)
    noise = X.noise_from_eta(p, eta, 0, scale)
    pxyz = oracle_noise(noise)
    sched = X.Schedule(noise, N, b0, b1, kind=kind)
    _, osyn = O.sample(d, pxyz, seed, shot0, n)
    refs = np.array([[O.greedy(d, pxyz, scale, seed, shot0 + s, i, 1, osyn[s])[0] for i in range(R)]
                     for s in range(n)])
    init = gpu_words(torch, labels_to_words(refs))
    out = X.anneal(code, sched, seed, shot0, init, want_cfg=True, want_final=True, per_warp=per_warp, order=order,
                   emin=emin)
    torch.cuda.synchronize()
    bE, fE = to_np(out["best_E"]), to_np(out["final_E"])
    bc = words_to_labels(to_np(out["best_cfg"]), d * d)
    fc = words_to_labels(to_np(out["final_cfg"]), d * d)
    LX, LZ = O.logicals(d)
    Ls = [0 * LX, LX, LX ^ LZ, LZ]
    for s in range(n):
        for i in range(R):
            for P in range(4):
                chain = ((shot0 + s) * R + i) * 4 + P
                if order == 0 and emin == 0:
                    ref = O.anneal_chain(d, pxyz, scale, kind, N, b0, b1, seed, chain, refs[s, i] ^ Ls[P])
                else:
                    ref = O.anneal_chain_variant(d, pxyz, scale, kind, N, b0, b1, seed, chain, refs[s, i] ^ Ls[P],
                                                 order, emin)
                assert bE[s, i, P] == ref["best_E"], (s, i, P)
                assert fE[s, i, P] == ref["final_E"], (s, i, P)
                assert np.array_equal(bc[s, i, P], ref["best"]), (s, i, P)
                assert np.array_equal(fc[s, i, P], ref["final"]), (s, i, P)


@pytest.mark.parametrize("d", [3, 5, 7, 9, 11, 13, 15, 17, 19, 21, 23, 25, 27, 29, 31])
def test_anneal_parity_every_distance(X, torch, d):
    # 3 shots x 5 restarts x 4 cosets = 60 chains: a ragged last warp
    anneal_case(X, torch, d, 0.18, 30, 3, 5, X.LINEAR, 24 if d < 21 else 10, 0.1, 6.0)


@pytest.mark.parametrize("d", [3, 5, 7, 11, 13, 17, 21, 25, 31])
def test_anneal_warp_per_chain_parity(X, torch, d):
    """One warp per chain (colour-parallel lanes) equals the oracle bit for bit."""
    anneal_case(X, torch, d, 0.18, 30, 3, 5, X.LINEAR, 24 if d < 21 else 10, 0.1, 6.0, per_warp=True)


@pytest.mark.parametrize("kind,N,b0,b1", [(0, 0, 0.1, 1.0), (0, 1, 0.4, 9.0), (0, 3, 0.0, 0.0),
                                          (0, 12, 1e6, 1e6), (1, 30, 0.9, 1.0), (0, 60, 0.05, 20.0)])
def test_anneal_parity_schedules(X, torch, kind, N, b0, b1):
    anneal_case(X, torch, 7, 0.2, 100, 4, 3, kind, N, b0, b1)
    anneal_case(X, torch, 9, 0.2, 100, 2, 3, kind, N, b0, b1, per_warp=True)


@pytest.mark.parametrize("d", [3, 5, 7, 11, 15, 17, 23, 31])
@pytest.mark.parametrize("order,emin", [(1, 0), (1, 1), (0, 1)])
def test_anneal_variant_parity(X, torch, d, order, emin):
    """Random-site Metropolis and per-attempt minima (the literal Alg. 2 /
    Alg. 3) equal the oracle's variants bit for bit."""
    anneal_case(X, torch, d, 0.18, 30, 3, 5, X.LINEAR, 16 if d < 21 else 6, 0.1, 6.0, order=order, emin=emin)


@pytest.mark.parametrize("order,emin", [(1, 1), (0, 1)])
def test_anneal_variant_paper_schedule(X, torch, order, emin):
    anneal_case(X, torch, 9, 0.12, 10, 2, 3, X.PAPER_LOG, 30, 0.9, 1.0, order=order, emin=emin, shot0=(1 << 31) + 3)


def test_anneal_variant_colour_equals_main_kernel(X, torch):
    """order 0 / emin 0 of the variant kernel is the main kernel's sweep: equal
    outputs on a batch of several CTAs with a ragged tail; emin 1 follows the
    same trajectory and never reports a higher minimum."""
    from paper_2509_17837_gb300 import api
    d, R, n = 11, 7, 37
    code = X.Code(d)
    noise = X.noise_from_eta(0.16, 100, 0, 1024)
    sched = X.Schedule(noise, 50, 0.05, 20.0)
    err, syn = X.sample_errors(code, noise, 5, 0, n)
    init, _ = X.greedy_init(code, noise, 5, 0, syn, R)
    a = X.anneal(code, sched, 5, 0, init, want_final=True)
    b = {k: torch.empty_like(v) for k, v in a.items()}
    api.call("xzzx_anneal_variant", code.handle, sched.handle, 5, 0, n, R, 0, 0, api._ptr(init), api._ptr(b["best_E"]),
             api._ptr(b["best_cfg"]), api._ptr(b["final_E"]), api._ptr(b["final_cfg"]), api._stream(None))
    v = X.anneal(code, sched, 5, 0, init, want_final=True, order=0, emin=1)
    torch.cuda.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k]), k
    assert bool((v["best_E"] <= a["best_E"]).all())
    assert torch.equal(v["final_E"], a["final_E"]) and torch.equal(v["final_cfg"], a["final_cfg"])


def test_anneal_variant_rejects_bad_modes(X, torch):
    code = X.Code(5)
    sched = X.Schedule(X.noise_from_eta(0.1, 1.0), 4, 0.1, 1.0)
    init = torch.zeros((1, 1, 2 * code.words), dtype=torch.int32, device="cuda")
    for order, emin in [(2, 0), (0, -1), (-1, 1)]:
        with pytest.raises(X.XzzxError):
            X.anneal(code, sched, 1, 0, init, order=order, emin=emin)
    with pytest.raises(ValueError):
        X.anneal(code, sched, 1, 0, init, order=1, per_warp=True)


def test_anneal_parity_large_chain_ids(X, torch):
    # chain ids above 2^32 use the high counter word
    anneal_case(X, torch, 5, 0.15, 10, 2, 3, X.LINEAR, 20, 0.1, 8.0, shot0=(1 << 31) + 7)


def test_anneal_parity_scale_4096(X, torch):
    anneal_case(X, torch, 9, 0.25, 1000, 2, 4, X.LINEAR, 40, 0.02, 30.0, scale=4096)


def decode_case(X, torch, d, p, eta, n, R, N, b0, b1, seed, shot0=0, scale=1024, want_best=True, mode=1):
    code = X.Code(d)
    noise = X.noise_from_eta(p, eta, 0, scale)
    pxyz = oracle_noise(noise)
    sched = X.Schedule(noise, N, b0, b1)
    oerr, osyn = O.sample(d, pxyz, seed, shot0, n)
    err, syn = X.sample_errors(code, noise, seed, shot0, n)
    out = X.decode_batch(code, noise, sched, seed, shot0, syn, R, randomised=mode, true_errors=err,
                         want_best_cfg=want_best)
    torch.cuda.synchronize()
    ref = O.decode(d, pxyz, scale, O.LINEAR, N, b0, b1, seed, shot0, R, osyn, oerr, randomised=mode)
    assert np.array_equal(to_np(out["cls"]), ref["cls"])
    assert np.array_equal(to_np(out["E4"]), ref["E4"])
    assert np.array_equal(words_to_labels(to_np(out["recovery"]), d * d), ref["recovery"])
    assert np.array_equal(to_np(out["fail"]), ref["fail"])
    if want_best:
        assert np.array_equal(words_to_labels(to_np(out["best_cfg"]), d * d), ref["best_cfg"])
    return ref


def test_decode_parity_d3_workload(X, torch):
    """The d = 3 workload in full: 1000 shots, 8 restarts, 200 sweeps, beta 0.1 -> 10."""
    ref = decode_case(X, torch, 3, 0.10, 10, 1000, 8, 200, 0.1, 10.0, 0xD3)
    assert 0 < ref["fail"].sum() < 200


@pytest.mark.parametrize("p", [0.10, 0.22])
def test_decode_parity_d11_workload_params(X, torch, p):
    """The d = 11 parameters (64 restarts, 1000 sweeps, beta 0.05 -> 20) on a few shots."""
    decode_case(X, torch, 11, p, 100, 3, 64, 1000, 0.05, 20.0, 0xD11, shot0=12345)


@pytest.mark.parametrize("d,n,R", [(5, 37, 7), (13, 5, 3), (25, 2, 2)])
def test_decode_parity_other_distances(X, torch, d, n, R):
    decode_case(X, torch, d, 0.15, 100, n, R, 50, 0.05, 20.0, 77)


@pytest.mark.parametrize("mode", [0, 2])
def test_decode_parity_init_modes(X, torch, mode):
    """Alg. 1 ("greedy same": deterministic greedy for every restart) and the
    boundary initializer, end to end."""
    decode_case(X, torch, 7, 0.15, 10, 40, 6, 80, 0.05, 20.0, 31, mode=mode)


def test_decode_batch_equals_pipeline(X, torch):
    d, n, R = 9, 50, 6
    code = X.Code(d)
    noise = X.noise_from_eta(0.17, 10)
    sched = X.Schedule(noise, 80, 0.1, 10.0)
    err, syn = X.sample_errors(code, noise, 9, 0, n)
    out = X.decode_batch(code, noise, sched, 9, 0, syn, R, true_errors=err, want_best_cfg=True)
    init, cbits = X.greedy_init(code, noise, 9, 0, syn, R)
    an = X.anneal(code, sched, 9, 0, init)
    red = X.decode_reduce(code, init, cbits, an["best_E"], an["best_cfg"], true_errors=err, want_best_cfg=True)
    torch.cuda.synchronize()
    for k in ("cls", "E4", "recovery", "best_cfg", "fail"):
        assert torch.equal(out[k], red[k]), k


def test_edge_cases(X, torch):
    d = 7
    code = X.Code(d)
    noise = X.noise_from_eta(0.1, 100)
    pxyz = oracle_noise(noise)
    sched = X.Schedule(noise, 30, 0.1, 10.0)
    # zero shots: nothing launched, nothing written
    empty = torch.zeros((0, code.syn_words), dtype=torch.int32, device="cuda")
    out = X.decode_batch(code, noise, sched, 1, 0, empty, 4)
    assert out["cls"].numel() == 0
    # empty and full syndromes, one restart
    osyn = np.stack([np.zeros(d * d - 1, np.uint8), np.ones(d * d - 1, np.uint8)])
    syn = gpu_words(torch, syn_bits_to_words(osyn))
    out = X.decode_batch(code, noise, sched, 1, 0, syn, 1, want_best_cfg=True)
    torch.cuda.synchronize()
    ref = O.decode(d, pxyz, noise.scale, O.LINEAR, 30, 0.1, 10.0, 1, 0, 1, osyn)
    assert np.array_equal(to_np(out["cls"]), ref["cls"])
    assert np.array_equal(to_np(out["E4"]), ref["E4"])
    assert np.array_equal(words_to_labels(to_np(out["recovery"]), d * d), ref["recovery"])
    assert to_np(out["cls"])[0] == 0 and to_np(out["E4"])[0, 0] == 0


def test_invalid_calls_fail_loudly(X, torch):
    import ctypes
    from paper_2509_17837_gb300._lib import XZZX_EINVAL, XzzxError, lib
    code = X.Code(5)
    noise = X.noise_from_eta(0.1, 100)
    sched = X.Schedule(noise, 10, 0.1, 10.0)
    err, syn = X.sample_errors(code, noise, 1, 0, 4)
    with pytest.raises(XzzxError) as e:
        X.decode_batch(code, noise, sched, 1, 0, syn, 0)             # restarts < 1
    assert e.value.status == XZZX_EINVAL
    out = dict(cls=torch.empty(4, dtype=torch.uint8, device="cuda"),
               E4=torch.empty((4, 4), dtype=torch.int32, device="cuda"),
               recovery=torch.empty((4, 2 * code.words), dtype=torch.int32, device="cuda"))
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = lib().xzzx_decode_batch(code.handle, ctypes.byref(noise), sched.handle, 1, 0, 4, 4, 1, p(syn), None,
                                 p(out["cls"]), p(out["E4"]), p(out["recovery"]), None, None, p(small),
                                 small.numel(), None)
    assert st == XZZX_EINVAL and b"workspace too small" in lib().xzzx_last_error()
    st = lib().xzzx_anneal(code.handle, sched.handle, 1, 0, 4, 2, None, p(out["E4"]), None, None, None, None)
    assert st == XZZX_EINVAL
    torch.cuda.synchronize()


def test_partition_independence(X, torch):
    """One call over shots [0, n) equals two calls over [0, k) and [k, n): the
    property that lets ranks (or serving slots) split shots freely."""
    d, n, k, R = 11, 90, 37, 8
    code = X.Code(d)
    noise = X.noise_from_eta(0.19, 100)
    sched = X.Schedule(noise, 100, 0.05, 20.0)
    err, syn = X.sample_errors(code, noise, 42, 1000, n)
    whole = X.decode_batch(code, noise, sched, 42, 1000, syn, R, true_errors=err, want_best_cfg=True)
    a = X.decode_batch(code, noise, sched, 42, 1000, syn[:k].contiguous(), R, true_errors=err[:k].contiguous(),
                       want_best_cfg=True)
    b = X.decode_batch(code, noise, sched, 42, 1000 + k, syn[k:].contiguous(), R,
                       true_errors=err[k:].contiguous(), want_best_cfg=True)
    torch.cuda.synchronize()
    for key in ("cls", "E4", "recovery", "best_cfg", "fail"):
        assert torch.equal(whole[key], torch.cat([a[key], b[key]])), key


@pytest.mark.parametrize("d,density,equal_weights", [(15, 0.5, False), (15, 0.6, False), (11, 0.5, True),
                                                     (15, 0.5, True)])
def test_greedy_parity_candidate_list_sizes(X, torch, d, density, equal_weights):
    """Colours just under and just over 64 vertices (the candidate-list path
    with its 64-wide sort, and the full scan), with equal X and Z weights so
    that many pairs tie and the random keys decide."""
    from inputs import random_syndromes
    code = X.Code(d)
    noise = X.make_noise(0.05, 0.05, 0.05) if equal_weights else X.make_noise(0.03, 0.05, 0.09)
    pxyz = oracle_noise(noise)
    osyn = random_syndromes(d * d - 1, 4, density, seed=100 + d)
    syn = gpu_words(torch, syn_bits_to_words(osyn))
    for randomised in (0, 1):
        init, cbits = X.greedy_init(code, noise, 9, 3, syn, 3, randomised=randomised)
        torch.cuda.synchronize()
        init = to_np(init)
        for s in range(4):
            for i in range(3):
                ref, _ = O.greedy(d, pxyz, noise.scale, 9, 3 + s, i, randomised, osyn[s])
                assert np.array_equal(words_to_labels(init[s, i], d * d), ref), (s, i, randomised)


@pytest.mark.parametrize("d,R,n", [(11, 64, 1024), (11, 64, 600), (7, 16, 4096), (9, 37, 1400)])
def test_greedy_restarts_per_warp_identical(X, torch, d, R, n):
    """A launch large enough that each greedy warp takes several restarts in
    turn (4 or 2; with 37 restarts the last group of each shot is partial)
    gives the references of small launches (one restart per warp), bit for
    bit, and sampled references equal the oracle."""
    code = X.Code(d)
    noise = X.noise_from_eta(0.16, 100.0)
    pxyz = oracle_noise(noise)
    err, syn = X.sample_errors(code, noise, 21, 0, n)
    big, big_cb = X.greedy_init(code, noise, 21, 0, syn, R)
    parts = [X.greedy_init(code, noise, 21, s0, syn[s0:s0 + 128], R) for s0 in range(0, n, 128)]
    torch.cuda.synchronize()
    assert torch.equal(big, torch.cat([p[0] for p in parts]))
    assert torch.equal(big_cb, torch.cat([p[1] for p in parts]))
    osyn = syn_words_to_bits(to_np(syn), d * d - 1)
    big = to_np(big)
    for s in (0, n // 2, n - 1):
        for i in (0, R // 2 + 1, R - 1):
            ref, _ = O.greedy(d, pxyz, noise.scale, 21, s, i, 1, osyn[s])
            assert np.array_equal(words_to_labels(big[s, i], d * d), ref), (s, i)
