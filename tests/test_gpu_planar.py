"""GPU parity on the planar layout (the paper's lattice): sampling, greedy
references, annealing in all four forms and the whole decoder, called through
the C ABI and compared with the oracle bit for bit on the same seeded inputs."""
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


def pxyz_of(noise):
    return (noise.px, noise.py, noise.pz)


@pytest.mark.parametrize("d,p,eta", [(3, 0.1, 10), (5, 0.2, 1.0), (11, 0.16, 5), (31, 0.25, 10)])
def test_planar_sample_parity(X, torch, d, p, eta):
    code = X.Code(d, X.LAYOUT_PLANAR)
    noise = X.noise_from_eta(p, eta, X.CONVENTION_PAPER)
    shot0, n = (1 << 33) + 5, 203
    err, syn = X.sample_errors(code, noise, 0xABC, shot0, n)
    torch.cuda.synchronize()
    oe, osyn = O.sample(O.planar(d), pxyz_of(noise), 0xABC, shot0, n)
    assert np.array_equal(words_to_labels(to_np(err), code.n_qubits), oe)
    assert np.array_equal(syn_words_to_bits(to_np(syn), code.n_stab), osyn)


@pytest.mark.parametrize("d,p,eta,n,R", [(3, 0.1, 10, 40, 8), (5, 0.2, 3, 30, 6), (11, 0.2, 5, 12, 5),
                                         (21, 0.15, 10, 4, 5), (31, 0.2, 10, 2, 4)])
@pytest.mark.parametrize("randomised", [1, 0, 2])
def test_planar_greedy_parity(X, torch, d, p, eta, n, R, randomised):
    cid = O.planar(d)
    code = X.Code(d, X.LAYOUT_PLANAR)
    noise = X.noise_from_eta(p, eta, X.CONVENTION_PAPER)
    pxyz = pxyz_of(noise)
    _, osyn = O.sample(cid, pxyz, 17, 100, n)
    syn = gpu_words(torch, syn_bits_to_words(osyn))
    init, cbits = X.greedy_init(code, noise, 17, 100, syn, R, randomised=randomised)
    torch.cuda.synchronize()
    init, cbits = to_np(init), to_np(cbits)
    for s in range(n):
        for i in range(R):
            ref, _ = O.greedy(cid, pxyz, noise.scale, 17, 100 + s, i, randomised, osyn[s])
            assert np.array_equal(words_to_labels(init[s, i], code.n_qubits), ref), (s, i)
            assert cbits[s, i] == O.class_bits(cid, ref)


@pytest.mark.parametrize("d,density", [(7, 0.5), (15, 0.3)])
def test_planar_greedy_unequal_weights(X, torch, d, density):
    from inputs import random_syndromes
    cid = O.planar(d)
    code = X.Code(d, X.LAYOUT_PLANAR)
    noise = X.make_noise(0.03, 0.05, 0.09)       # Wt_x != Wt_z
    osyn = random_syndromes(code.n_stab, 4, density, seed=d)
    syn = gpu_words(torch, syn_bits_to_words(osyn))
    init, _ = X.greedy_init(code, noise, 5, 7, syn, 3)
    torch.cuda.synchronize()
    init = to_np(init)
    for s in range(4):
        for i in range(3):
            ref, _ = O.greedy(cid, pxyz_of(noise), noise.scale, 5, 7 + s, i, 1, osyn[s])
            assert np.array_equal(words_to_labels(init[s, i], code.n_qubits), ref)


def planar_anneal_case(X, torch, d, p, eta, n, R, kind, N, b0, b1, order=0, emin=0, seed=3, shot0=11):
    cid = O.planar(d)
    code = X.Code(d, X.LAYOUT_PLANAR)
    noise = X.noise_from_eta(p, eta, X.CONVENTION_PAPER)
    pxyz = pxyz_of(noise)
    sched = X.Schedule(noise, N, b0, b1, kind=kind)
    _, osyn = O.sample(cid, pxyz, seed, shot0, n)
    refs = np.array([[O.greedy(cid, pxyz, noise.scale, seed, shot0 + s, i, 1, osyn[s])[0] for i in range(R)]
                     for s in range(n)])
    init = gpu_words(torch, labels_to_words(refs))
    out = X.anneal(code, sched, seed, shot0, init, want_cfg=True, want_final=True, order=order, emin=emin)
    torch.cuda.synchronize()
    nq = code.n_qubits
    bE, fE = to_np(out["best_E"]), to_np(out["final_E"])
    bc, fc = words_to_labels(to_np(out["best_cfg"]), nq), words_to_labels(to_np(out["final_cfg"]), nq)
    LX, LZ = O.logicals(cid)
    Ls = [0 * LX, LX, LX ^ LZ, LZ]
    for s in range(n):
        for i in range(R):
            for P in range(4):
                chain = ((shot0 + s) * R + i) * 4 + P
                ref = O.anneal_chain_variant(cid, pxyz, noise.scale, kind, N, b0, b1, seed, chain,
                                             refs[s, i] ^ Ls[P], order, emin)
                assert bE[s, i, P] == ref["best_E"], (s, i, P)
                assert fE[s, i, P] == ref["final_E"], (s, i, P)
                assert np.array_equal(bc[s, i, P], ref["best"]), (s, i, P)
                assert np.array_equal(fc[s, i, P], ref["final"]), (s, i, P)


@pytest.mark.parametrize("d", [3, 5, 7, 11, 15, 17, 23, 31])
@pytest.mark.parametrize("order,emin", [(0, 0), (1, 0), (1, 1), (0, 1)])
def test_planar_anneal_parity(X, torch, d, order, emin):
    # 3 shots x 5 restarts x 4 cosets = 60 chains: a ragged last warp
    planar_anneal_case(X, torch, d, 0.18, 5, 3, 5, X.LINEAR, 16 if d < 21 else 6, 0.1, 6.0, order, emin)


@pytest.mark.parametrize("kind,N,b0,b1", [(0, 0, 0.1, 1.0), (0, 1, 0.4, 9.0), (1, 30, 0.9, 1.0), (0, 12, 1e6, 1e6)])
def test_planar_anneal_schedules(X, torch, kind, N, b0, b1):
    planar_anneal_case(X, torch, 9, 0.12, 10, 2, 3, kind, N, b0, b1)
    planar_anneal_case(X, torch, 5, 0.2, 1.0, 2, 3, kind, N, b0, b1, order=1, emin=1)


def test_planar_chain_ids_above_2_32(X, torch):
    planar_anneal_case(X, torch, 5, 0.15, 10, 2, 3, X.LINEAR, 20, 0.1, 8.0, shot0=(1 << 31) + 7)


@pytest.mark.parametrize("d,n,R,N,mode", [(3, 300, 8, 100, 1), (5, 60, 6, 60, 1), (7, 20, 4, 40, 0),
                                          (9, 16, 4, 30, 2)])
def test_planar_decode_parity(X, torch, d, n, R, N, mode):
    cid = O.planar(d)
    code = X.Code(d, X.LAYOUT_PLANAR)
    noise = X.noise_from_eta(0.12, 10, X.CONVENTION_PAPER)
    pxyz = pxyz_of(noise)
    sched = X.Schedule(noise, N, 0.9, 1.0, kind=X.PAPER_LOG)
    seed, shot0 = 0xB0 + d, 3
    oerr, osyn = O.sample(cid, pxyz, seed, shot0, n)
    err, syn = X.sample_errors(code, noise, seed, shot0, n)
    out = X.decode_batch(code, noise, sched, seed, shot0, syn, R, randomised=mode, true_errors=err,
                         want_best_cfg=True)
    torch.cuda.synchronize()
    ref = O.decode(cid, pxyz, noise.scale, O.PAPER_LOG, N, 0.9, 1.0, seed, shot0, R, osyn, oerr, randomised=mode)
    nq = code.n_qubits
    assert np.array_equal(to_np(out["cls"]), ref["cls"])
    assert np.array_equal(to_np(out["E4"]), ref["E4"])
    assert np.array_equal(words_to_labels(to_np(out["recovery"]), nq), ref["recovery"])
    assert np.array_equal(words_to_labels(to_np(out["best_cfg"]), nq), ref["best_cfg"])
    assert np.array_equal(to_np(out["fail"]), ref["fail"])


def test_planar_default_anneal_is_colour_sweep(X, torch):
    """xzzx_anneal on a planar code is the colour sweep with per-phase minima:
    equal to xzzx_anneal_variant (0, 0) on several CTAs with a ragged tail."""
    from paper_2509_17837_gb300 import api
    d, R, n = 9, 7, 37
    code = X.Code(d, X.LAYOUT_PLANAR)
    noise = X.noise_from_eta(0.16, 5, X.CONVENTION_PAPER)
    sched = X.Schedule(noise, 40, 0.05, 20.0)
    err, syn = X.sample_errors(code, noise, 5, 0, n)
    init, _ = X.greedy_init(code, noise, 5, 0, syn, R)
    a = X.anneal(code, sched, 5, 0, init, want_final=True)
    b = {k: torch.empty_like(v) for k, v in a.items()}
    api.call("xzzx_anneal_variant", code.handle, sched.handle, 5, 0, n, R, 0, 0, api._ptr(init),
             api._ptr(b["best_E"]), api._ptr(b["best_cfg"]), api._ptr(b["final_E"]), api._ptr(b["final_cfg"]),
             api._stream(None))
    torch.cuda.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_planar_rotated_only_paths_refuse(X, torch):
    from paper_2509_17837_gb300._lib import XZZX_EUNSUPPORTED, XzzxError
    code = X.Code(5, X.LAYOUT_PLANAR)
    noise = X.noise_from_eta(0.1, 1.0)
    sched = X.Schedule(noise, 4, 0.1, 1.0)
    init = torch.zeros((1, 1, 2 * code.words), dtype=torch.int32, device="cuda")
    with pytest.raises(XzzxError) as e:
        X.anneal(code, sched, 1, 0, init, per_warp=True)
    assert e.value.status == XZZX_EUNSUPPORTED
    syn = torch.zeros((2, code.syn_words), dtype=torch.int32, device="cuda")
    with pytest.raises(XzzxError) as e:
        X.Batch([dict(code=code, noise=noise, sched=sched, shot0=0, syndromes=syn, restarts=2)], seed=1)
    assert e.value.status == XZZX_EUNSUPPORTED
