"""The d = 5 accuracy bar of the simulated-annealing decoder (Eq. min_energy,
Alg. 7), checked on 1000 seeded shots against exact coset minima.

For every shot the exact E^min_P of the four cosets of the greedy reference
R_1 is found by enumerating all 2^24 elements of the stabilizer group in
Gray-code order.  The noise point is the middle of the d = 11 benchmark sweep
(p = 0.16, Y-biased eta = 100) and the annealing schedule is that
benchmark's: 64 restarts, 1000 sweeps, linear beta 0.05 -> 20.
Simulated annealing must never report an energy below the exact minimum of its coset,
and its lowest coset energy must equal the exact global minimum on at least
99.9% of shots.  The share of shots whose decision P* equals the exact
argmin is reported (the two can differ only where SA misses a minimum or the
exact minima tie).  Logical failures of SA equal those of the exact
minimum-energy decision, and are far fewer than those of the decision taken
from the greedy initial configurations alone (0 sweeps).

The shots are sharded over every host core (about 0.35 s of enumeration per
shot on one core).
"""
import math

import numpy as np
import pytest

import oracle_pool

D5 = dict(d=5, p=0.16, eta=100, scale=1024, shots=1000, restarts=64, sweeps=1000, b0=0.05, b1=20.0, seed=0xD5)


@pytest.mark.slow
def test_sa_against_bruteforce_d5_1000_shots():
    c = D5
    tasks = [(c, a, b) for a, b in oracle_pool.chunks(0, c["shots"], 4 * oracle_pool.n_workers(c["shots"]))]
    parts = oracle_pool.run(oracle_pool.bruteforce_vs_sa, tasks)
    sa = np.concatenate([p[0] for p in parts])
    exact = np.concatenate([p[1] for p in parts])
    cls = np.concatenate([p[2] for p in parts])
    assert sa.shape == exact.shape == (c["shots"], 4)
    assert (sa >= exact).all(), np.nonzero((sa < exact).any(1))[0][:10]     # never below E^min_P
    hits = int((sa.min(1) == exact.min(1)).sum())
    assert hits >= math.ceil(0.999 * c["shots"]), hits
    # P* against the exact argmin (first of I, X, Y, Z on ties)
    same_decision = int((cls == exact.argmin(1)).sum())
    print("d=5 brute force: %d/%d shots at the global minimum, %d/%d with the exact decision"
          % (hits, c["shots"], same_decision, c["shots"]))
    ties = int(((exact == exact.min(1, keepdims=True)).sum(1) > 1).sum())
    assert same_decision >= hits - ties
    # logical failures: SA fails exactly where the exact minimum-energy decision
    # fails, and both fail far less often than the decision taken from the
    # greedy initial configurations alone (Sec. "Logical error rates")
    sa_fail = np.concatenate([p[3] for p in parts])
    med_fail = np.concatenate([p[4] for p in parts])
    none_fail = np.concatenate([p[5] for p in parts])
    print("failures: SA %d, exact minimum energy %d, initial configurations only %d"
          % (sa_fail.sum(), med_fail.sum(), none_fail.sum()))
    assert np.array_equal(sa_fail[cls == exact.argmin(1)], med_fail[cls == exact.argmin(1)])
    assert sa_fail.sum() < 0.2 * none_fail.sum()
