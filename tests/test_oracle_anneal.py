"""Pins of the oracle's simulated annealing (Algs. 2, 3) and decoder (Alg. 7).

* Every move multiplies by a generator, so the syndrome never changes
  (Alg. 3 and the footnote on bit flips), the coset never changes
  (Eq. coset_decomp), and the tracked energy equals Eq. energy recomputed.
* beta = 0 accepts every move: one sweep multiplies by every generator once.
* A huge beta accepts only dE <= 0: the energy never rises.
* At fixed beta the colour sweep samples exp(-beta H) over the coset
  (Eq. pi_beta_def): the energy histogram matches the exact distribution
  enumerated over all 2^8 configurations of a d = 3 coset.
* SA never undercuts the exact coset minima E^min_P of Eq. min_energy found by
  enumerating the stabilizer group, and reaches the global minimum on at least
  99.9% of d = 3 shots of the d = 3 workload (and on sampled d = 5 shots).
* The decoder's outputs obey Eq. determine_P_from_E and the failure test of
  Sec. "Simulation setting"; a distance-d code under equal weights corrects
  every single-qubit error.
"""
import math

import numpy as np
import pytest

import oracle as O
from codehelp import generators_from_syndromes

D3 = dict(d=3, p=0.10, eta=10, scale=1024, shots=1000, restarts=8, sweeps=200, b0=0.1, b1=10.0, seed=0xD3)


def energy(W4, cfg):
    return int(np.asarray(W4, np.int64)[cfg].sum())


@pytest.mark.parametrize("d,p,eta", [(3, 0.1, 10), (5, 0.15, 100), (11, 0.2, 100), (O.planar(3), 0.1, 10),
                                     (O.planar(7), 0.2, 100)])
def test_chain_invariants(d, p, eta):
    pxyz = O.noise_from_eta(p, eta)
    W4, _ = O.make_noise(*pxyz, 1024)
    err, syn = O.sample(d, pxyz, 11, 0, 6)
    LX, LZ = O.logicals(d)
    for s in range(6):
        R, _ = O.greedy(d, pxyz, 1024, 11, s, 0, 1, syn[s])
        for P, L in enumerate([0 * LX, LX, LX ^ LZ, LZ]):
            init = R ^ L
            out = O.anneal_chain(d, pxyz, 1024, O.LINEAR, 40, 0.1, 5.0, 11, 4 * s + P, init)
            for key in ("best", "final"):
                assert np.array_equal(O.syndrome(d, out[key]), syn[s])
                assert O.class_bits(d, out[key] ^ init) == 0   # same coset as the start
                assert out[key + "_E"] == energy(W4, out[key])
            assert out["best_E"] <= min(out["final_E"], energy(W4, init))


def test_beta_zero_applies_every_generator():
    d = 5
    pxyz = O.noise_from_eta(0.1, 10)
    G = generators_from_syndromes(d)
    prod = np.bitwise_xor.reduce(G, axis=0)
    init = np.zeros(O.code_sizes(d)[0], np.uint8)
    one = O.anneal_chain(d, pxyz, 1024, O.LINEAR, 1, 0.0, 0.0, 3, 0, init)
    assert np.array_equal(one["final"], prod)
    two = O.anneal_chain(d, pxyz, 1024, O.LINEAR, 2, 0.0, 0.0, 3, 0, init)
    assert np.array_equal(two["final"], init)


def test_huge_beta_is_pure_descent():
    d = 7
    pxyz = O.noise_from_eta(0.2, 100)
    err, syn = O.sample(d, pxyz, 5, 0, 10)
    for s in range(10):
        out = O.anneal_chain(d, pxyz, 1024, O.LINEAR, 30, 1e6, 1e6, 5, s, err[s], trace=True)
        tr = out["trace_E"]
        assert (np.diff(tr) <= 0).all()
        assert out["best_E"] == out["final_E"] == tr[-1]


@pytest.mark.parametrize("d,p,eta,beta", [(3, 0.25, 3, 0.15), (3, 0.25, 3, 0.35), (3, 0.3, 1.0, 1.0),
                                          (O.planar(3), 0.25, 3, 0.35), (O.planar(3), 0.3, 1.0, 1.0)])
def test_detailed_balance_d3(d, p, eta, beta):
    pxyz = O.noise_from_eta(p, eta)
    W4, _ = O.make_noise(*pxyz, 1024)
    err, syn = O.sample(d, pxyz, 21, 3, 1)
    start = err[0]
    levels = O.coset_energies(d, pxyz, 1024, start)
    vals, g = np.unique(levels, return_counts=True)
    w = g * np.exp(-beta * (vals - vals.min()) / 1024.0)
    exact = w / w.sum()
    n_sweeps, thin = 60000, 3
    out = O.anneal_chain(d, pxyz, 1024, O.LINEAR, n_sweeps, beta, beta, 99, 7, start, trace=True)
    sample = out["trace_E"][1000::thin]
    idx = np.searchsorted(vals, sample)
    assert np.array_equal(vals[idx], sample)     # only coset energies are visited
    counts = np.bincount(idx, minlength=len(vals))
    n = counts.sum()
    # merge sparse levels into one bin so every expected count is >= 20
    order = np.argsort(-exact)
    chi2, dof, acc_e, acc_c = 0.0, -1, 0.0, 0
    for i in order:
        acc_e += n * exact[i]
        acc_c += counts[i]
        if acc_e >= 20:
            chi2 += (acc_c - acc_e) ** 2 / acc_e
            dof += 1
            acc_e, acc_c = 0.0, 0
    assert dof >= 3
    # samples are mildly correlated: allow a generous margin over dof
    assert chi2 < 3 * dof + 10 * math.sqrt(2 * dof), (chi2, dof)


def run_d3_workload(shots):
    c = D3
    pxyz = O.noise_from_eta(c["p"], c["eta"])
    err, syn = O.sample(c["d"], pxyz, c["seed"], 0, shots)
    out = O.decode(c["d"], pxyz, c["scale"], O.LINEAR, c["sweeps"], c["b0"], c["b1"], c["seed"], 0,
                   c["restarts"], syn, err, want_chains=True)
    return pxyz, err, syn, out


def test_sa_against_bruteforce_d3():
    c = D3
    pxyz, err, syn, out = run_d3_workload(c["shots"])
    LX, LZ = O.logicals(3)
    hits = 0
    for s in range(c["shots"]):
        R1, _ = O.greedy(3, pxyz, c["scale"], c["seed"], s, 0, 1, syn[s])
        bf = O.bruteforce(3, pxyz, c["scale"], R1)
        assert (out["E4"][s] >= bf).all()                 # SA never undercuts E^min_P
        hits += out["E4"][s].min() == bf.min()
    assert hits >= math.ceil(0.999 * c["shots"])


def test_sa_against_bruteforce_d5():
    d, scale = 5, 1024
    pxyz = O.noise_from_eta(0.12, 10)
    err, syn = O.sample(d, pxyz, 0xD5, 0, 12)
    out = O.decode(d, pxyz, scale, O.LINEAR, 300, 0.1, 10.0, 0xD5, 0, 8, syn, err)
    for s in range(12):
        R1, _ = O.greedy(d, pxyz, scale, 0xD5, s, 0, 1, syn[s])
        bf = O.bruteforce(d, pxyz, scale, R1)
        assert (out["E4"][s] >= bf).all()
        assert out["E4"][s].min() == bf.min()


def test_decode_outputs_consistent():
    c = D3
    pxyz, err, syn, out = run_d3_workload(200)
    W4, _ = O.make_noise(*pxyz, c["scale"])
    LX, LZ = O.logicals(3)
    Ls = [0 * LX, LX, LX ^ LZ, LZ]
    for s in range(200):
        cls = int(out["cls"][s])
        E4 = out["E4"][s]
        assert E4[cls] == E4.min() and all(E4[P] > E4[cls] for P in range(cls))  # ties -> I<X<Y<Z
        R1, _ = O.greedy(3, pxyz, c["scale"], c["seed"], s, 0, 1, syn[s])
        assert np.array_equal(out["recovery"][s], R1 ^ Ls[cls])               # R_1 L_{P*}
        assert np.array_equal(O.syndrome(3, out["recovery"][s]), syn[s])
        best = out["best_cfg"][s]
        assert np.array_equal(O.syndrome(3, best), syn[s])
        assert energy(W4, best) == E4[cls]
        assert O.class_bits(3, best ^ out["recovery"][s]) == 0
        assert out["fail"][s] == (O.class_bits(3, err[s] ^ out["recovery"][s]) != 0)
        # chain (i, P) belongs to coset Q_i P; its minimum feeds E_{Q_i P}
        ce = out["chain_E"][s].reshape(-1, 4)
        to_bits, to_idx = [0, 1, 3, 2], [0, 1, 3, 2]
        for P in range(4):
            m = min(ce[i, Pc] for i in range(ce.shape[0]) for Pc in range(4)
                    if to_idx[out["q_bits"][s][i] ^ to_bits[Pc]] == P)
            assert m == E4[P]


@pytest.mark.parametrize("d", [3, 5, O.planar(3), O.planar(5)])
def test_single_errors_are_corrected(d):
    pxyz = O.noise_from_eta(0.05, 1.0, O.PAPER_ETA)     # equal weights
    nq, ns, _ = O.code_sizes(d)
    errs = []
    for q in range(nq):
        for lab in (1, 2, 3):
            e = np.zeros(nq, np.uint8)
            e[q] = lab
            errs.append(e)
    errs = np.array(errs)
    syn = np.array([O.syndrome(d, e) for e in errs])
    out = O.decode(d, pxyz, 1024, O.LINEAR, 60, 0.2, 8.0, 4, 0, 4, syn, errs)
    assert out["fail"].sum() == 0


def test_annealing_beats_initialisation():
    """P_L falls once SA runs on top of the greedy start (Sec. "Logical error rates")."""
    d = 5
    pxyz = O.noise_from_eta(0.12, 1.0, O.PAPER_ETA)
    err, syn = O.sample(d, pxyz, 8, 0, 800)
    none = O.decode(d, pxyz, 1024, O.LINEAR, 0, 0.1, 10.0, 8, 0, 4, syn, err)
    sa = O.decode(d, pxyz, 1024, O.LINEAR, 100, 0.1, 10.0, 8, 0, 4, syn, err)
    assert sa["fail"].sum() < none["fail"].sum()
    assert (sa["E4"].min(1) <= none["E4"].min(1)).all()


def test_coset_ties_break_in_pauli_order():
    """When two cosets share the minimum energy, P* is the first in I, X, Y, Z
    order (the tie rule adopted where Eq. determine_P_from_E is silent).  Ties
    are found by exact enumeration, so the check does not rely on SA luck."""
    d = 3
    pxyz = O.noise_from_eta(0.3, 1.0, O.PAPER_ETA)   # equal weights: many ties
    err, syn = O.sample(d, pxyz, 31, 0, 300)
    out = O.decode(d, pxyz, 1024, O.LINEAR, 150, 0.1, 10.0, 31, 0, 8, syn, err)
    n_ties = 0
    for s in range(300):
        R1, _ = O.greedy(d, pxyz, 1024, 31, s, 0, 1, syn[s])
        bf = O.bruteforce(d, pxyz, 1024, R1)
        if not np.array_equal(out["E4"][s], bf):
            continue
        winners = np.nonzero(bf == bf.min())[0]
        if len(winners) > 1:
            n_ties += 1
            assert out["cls"][s] == winners[0]
    assert n_ties >= 10
