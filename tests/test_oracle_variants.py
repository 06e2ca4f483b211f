"""Pins of the paper-faithful variants kept beside the adopted readings.

* "Boundary" initializer (Sec. "Effect of initial error configuration"):
  reproduces the syndrome, weighs the sum of the defects' boundary distances
  (networkx-pinned in test_oracle_greedy), and is one boundary walk per defect.
* "Greedy (same)" (Alg. 1): the deterministic greedy gives every restart the
  same reference.
* Per-attempt minimum (Alg. 2 as printed) on the same trajectory: same moves,
  same final state, a minimum never above the per-colour-phase minimum and
  equal to the lowest energy visited.
* Random-site Metropolis (Alg. 3 as printed): keeps syndrome and coset,
  samples exp(-beta H) at fixed beta (d = 3 chi-square against exact
  enumeration), and anneals to the brute-force minimum like the colour sweep.
"""
import math

import numpy as np
import pytest

import oracle as O
from inputs import random_syndromes


@pytest.mark.parametrize("d", [3, 5, 11, 31])
def test_boundary_initializer(d):
    pxyz = O.noise_from_eta(0.15, 10)
    wb = O.boundary_distance(d, pxyz, 1024)
    _, ns, _ = O.code_sizes(d)
    for s, syn in enumerate(random_syndromes(ns, 6, 0.2, seed=d)):
        R, w = O.greedy(d, pxyz, 1024, 1, s, 0, O.INIT_BOUNDARY, syn)
        assert np.array_equal(O.syndrome(d, R), syn)
        assert w == int(wb[syn == 1].sum())
        ref = np.zeros(d * d, np.uint8)
        for f in np.nonzero(syn)[0]:
            ref ^= O.walk_boundary(d, pxyz, 1024, int(f))
        assert np.array_equal(R, ref)


def test_greedy_same_gives_identical_references():
    d = 7
    pxyz = O.noise_from_eta(0.2, 10)
    _, syn = O.sample(d, pxyz, 4, 0, 5)
    for s in range(5):
        refs = {O.greedy(d, pxyz, 1024, 4, s, i, O.INIT_GREEDY, syn[s])[0].tobytes() for i in range(6)}
        assert len(refs) == 1


@pytest.mark.parametrize("order", [O.ORDER_COLOUR, O.ORDER_RANDOM_SITE])
def test_per_attempt_minimum_on_the_same_trajectory(order):
    d = 7
    pxyz = O.noise_from_eta(0.2, 100)
    W4, _ = O.make_noise(*pxyz, 1024)
    err, syn = O.sample(d, pxyz, 6, 0, 8)
    for s in range(8):
        a = O.anneal_chain_variant(d, pxyz, 1024, O.LINEAR, 50, 0.1, 8.0, 6, s, err[s], order, O.EMIN_PER_PHASE,
                                   trace=True)
        b = O.anneal_chain_variant(d, pxyz, 1024, O.LINEAR, 50, 0.1, 8.0, 6, s, err[s], order, O.EMIN_PER_ATTEMPT,
                                   trace=True)
        assert np.array_equal(a["final"], b["final"]) and np.array_equal(a["trace_E"], b["trace_E"])
        assert b["best_E"] <= a["best_E"]
        assert b["best_E"] <= min(int(a["trace_E"].min()), int(W4[err[s]].sum()))
        assert int(W4[b["best"]].sum()) == b["best_E"]
        assert np.array_equal(O.syndrome(d, b["best"]), syn[s])


def test_colour_sweep_variant_matches_default():
    d = 5
    pxyz = O.noise_from_eta(0.15, 10)
    err, _ = O.sample(d, pxyz, 2, 0, 4)
    for s in range(4):
        a = O.anneal_chain(d, pxyz, 1024, O.LINEAR, 30, 0.1, 5.0, 2, s, err[s])
        b = O.anneal_chain_variant(d, pxyz, 1024, O.LINEAR, 30, 0.1, 5.0, 2, s, err[s], O.ORDER_COLOUR,
                                   O.EMIN_PER_PHASE)
        assert a["best_E"] == b["best_E"] and np.array_equal(a["best"], b["best"])


def test_random_site_detailed_balance_d3():
    d, beta = 3, 0.35
    pxyz = O.noise_from_eta(0.25, 3)
    err, _ = O.sample(d, pxyz, 21, 3, 1)
    levels = O.coset_energies(d, pxyz, 1024, err[0])
    vals, g = np.unique(levels, return_counts=True)
    w = g * np.exp(-beta * (vals - vals.min()) / 1024.0)
    exact = w / w.sum()
    out = O.anneal_chain_variant(d, pxyz, 1024, O.LINEAR, 60000, beta, beta, 5, 9, err[0], O.ORDER_RANDOM_SITE,
                                 O.EMIN_PER_PHASE, trace=True)
    sample = out["trace_E"][1000::3]
    idx = np.searchsorted(vals, sample)
    assert np.array_equal(vals[idx], sample)
    counts = np.bincount(idx, minlength=len(vals))
    n = counts.sum()
    chi2, dof, acc_e, acc_c = 0.0, -1, 0.0, 0
    for i in np.argsort(-exact):
        acc_e += n * exact[i]
        acc_c += counts[i]
        if acc_e >= 20:
            chi2 += (acc_c - acc_e) ** 2 / acc_e
            dof += 1
            acc_e, acc_c = 0.0, 0
    assert dof >= 3 and chi2 < 3 * dof + 10 * math.sqrt(2 * dof), (chi2, dof)


def test_random_site_reaches_bruteforce_minimum_d3():
    d, R = 3, 8
    pxyz = O.noise_from_eta(0.10, 10)
    LX, LZ = O.logicals(d)
    Ls = [0 * LX, LX, LX ^ LZ, LZ]
    err, syn = O.sample(d, pxyz, 0xD3, 0, 150)
    hits = 0
    for s in range(150):
        R1, _ = O.greedy(d, pxyz, 1024, 0xD3, s, 0, 1, syn[s])
        bf = O.bruteforce(d, pxyz, 1024, R1)
        best = min(O.anneal_chain_variant(d, pxyz, 1024, O.LINEAR, 200, 0.1, 10.0, 0xD3, (s * R + i) * 4 + P,
                                          O.greedy(d, pxyz, 1024, 0xD3, s, i, 1, syn[s])[0] ^ Ls[P],
                                          O.ORDER_RANDOM_SITE, O.EMIN_PER_ATTEMPT)["best_E"]
                   for i in range(R) for P in range(4))
        assert best >= bf.min()
        hits += best == bf.min()
    assert hits >= 148
