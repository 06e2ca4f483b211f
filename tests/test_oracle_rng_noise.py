"""Pins of the oracle's generator, noise model, energies and thresholds.

* Philox4x32-10 against the known-answer vectors published with the generator
  (Salmon et al., SC'11; Random123 kat_vectors), plus uniformity.
* Sampling against Eq. noise_map: per-qubit X/Y/Z frequencies within binomial
  bounds; the bias conventions of Sec. "Simulation setting".
* Integer energies against Eq. prob_C: H(C)/scale equals -ln(Pr(C)/(1-p)^N)
  computed from the product of per-qubit probabilities, to within the rounding
  of the N weights.
* Acceptance thresholds against an independent 60-digit evaluation of
  2^32 exp(-beta dE / scale) (mpmath), and the schedule endpoints of Eq. beta_i.
"""
import math

import numpy as np
import pytest

import oracle as O
import golden_data
from inputs import random_paulis

KAT = golden_data.philox_kat()


@pytest.mark.parametrize("key,ctr,out", KAT)
def test_philox_known_answers(key, ctr, out):
    assert [int(x) for x in O.philox(key, ctr)] == out


def test_kat_fixture_complete():
    assert len(KAT) == 3


@pytest.mark.parametrize("p,eta,scale,wx,wy,wt", golden_data.weight_table())
def test_weights_equal_printed_table(p, eta, scale, wx, wy, wt):
    """The oracle's integer weights equal the stored values of Eq. coeff_in_energy
    (W_X = W_Z, W_Y) and Eq. coeff_in_distance (matching weights)."""
    W4, Wt = O.make_noise(*O.noise_from_eta(p, eta), scale)
    assert [int(x) for x in W4] == [0, wx, wx, wy]       # labels I, Z, X, Y
    assert [int(x) for x in Wt] == [wt, wt]


def test_philox_uniform():
    vals = np.concatenate([O.philox(12345, [i, 7, 9, 3]) for i in range(4096)]).astype(np.uint64)
    hist = np.bincount((vals >> np.uint64(28)).astype(np.int64), minlength=16)
    exp = len(vals) / 16
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 45.0  # 15 dof; p ~ 1e-4
    bits = np.unpackbits(vals.astype(np.uint32).view(np.uint8))
    assert abs(bits.mean() - 0.5) < 5 * 0.5 / math.sqrt(bits.size)


def test_bias_conventions():
    px, py, pz = O.noise_from_eta(0.1, 10, O.Y_OVER_XZ_ETA)
    assert math.isclose(py, 0.1 * 10 / 11) and math.isclose(px, 0.1 / 22) and px == pz
    assert math.isclose(px + py + pz, 0.1)
    px, py, pz = O.noise_from_eta(0.3, 1.0, O.PAPER_ETA)   # eta = 1 is depolarizing
    assert math.isclose(px, 0.1) and math.isclose(py, 0.1) and math.isclose(pz, 0.1)


@pytest.mark.parametrize("p,eta", [(0.10, 10), (0.22, 100), (0.3, 1.0)])
def test_sampling_frequencies(p, eta):
    pxyz = O.noise_from_eta(p, eta)
    err, syn = O.sample(11, pxyz, 99, 5, 3000)
    n = err.size
    for lab, prob in ((2, pxyz[0]), (3, pxyz[1]), (1, pxyz[2])):
        k = (err == lab).sum()
        sigma = math.sqrt(n * prob * (1 - prob))
        assert abs(k - n * prob) < 5 * sigma + 1
    # the syndrome rows are the syndromes of the sampled errors
    for s in range(0, 3000, 97):
        assert np.array_equal(O.syndrome(11, err[s]), syn[s])


def test_sampling_counter_independence():
    pxyz = O.noise_from_eta(0.2, 1.0)
    e1, _ = O.sample(5, pxyz, 1, 0, 10)
    e2, _ = O.sample(5, pxyz, 1, 3, 4)
    assert np.array_equal(e1[3:7], e2)        # a shot depends only on (seed, shot)
    e3, _ = O.sample(5, pxyz, 2, 0, 10)
    assert not np.array_equal(e1, e3)


def test_syndrome_linear_and_generator_invariant():
    d = 7
    A = random_paulis(d * d, 20, seed=3)
    B = random_paulis(d * d, 20, seed=4)
    for a, b in zip(A, B):
        assert np.array_equal(O.syndrome(d, a ^ b), O.syndrome(d, a) ^ O.syndrome(d, b))


@pytest.mark.parametrize("p,eta,scale", [(0.10, 10, 1024), (0.10, 100, 1024), (0.22, 100, 1024),
                                         (0.15, 1000, 4096), (0.30, 1000, 4096), (0.05, 0.5, 1024)])
def test_energy_matches_configuration_probability(p, eta, scale):
    pxyz = O.noise_from_eta(p, eta)
    W4, Wt = O.make_noise(*pxyz, scale)
    ptot = sum(pxyz)
    prob = {0: 1 - ptot, 2: pxyz[0], 3: pxyz[1], 1: pxyz[2]}   # I, X, Y, Z by two-bit label
    cfgs = random_paulis(121, 50, seed=int(p * 1000 + eta * 10))
    for c in cfgs:
        logpr = sum(math.log(prob[int(s)]) for s in c)                  # Eq. prob_C, first line
        nat = -(logpr - len(c) * math.log(1 - ptot))                     # -ln pi(C)
        H = int(W4[c].sum())
        assert abs(H / scale - nat) <= 0.5 * np.count_nonzero(c) / scale + 1e-9
    # Eq. coeff_in_distance: the matching weights see X and Z components
    for w, pt in ((Wt[0], pxyz[0] + pxyz[1]), (Wt[1], pxyz[2] + pxyz[1])):
        assert abs(w / scale + math.log(pt / (1 - ptot))) <= 0.5 / scale


def test_weight_ordering_y_bias():
    W4, Wt = O.make_noise(*O.noise_from_eta(0.1, 100), 1024)
    assert W4[0] == 0 and W4[3] < W4[2] == W4[1]
    assert Wt[0] == Wt[1] <= W4[3]


def test_schedule_endpoints():
    for kind in (O.LINEAR, O.PAPER_LOG):
        assert O.beta_at(kind, 1000, 0.05, 20.0, 0) == pytest.approx(0.05)
        assert O.beta_at(kind, 1000, 0.05, 20.0, 999) == pytest.approx(20.0)
    b = [O.beta_at(O.LINEAR, 11, 1.0, 2.0, t) for t in range(11)]
    assert np.allclose(np.diff(b), 0.1)
    # Eq. beta_i: beta_init (1 + gamma ln i), gamma = (beta_final/beta_init - 1)/ln N
    N = 100
    g = (1.0 / 0.9 - 1) / math.log(N)
    for i in (1, 2, 10, 57, 100):
        assert O.beta_at(O.PAPER_LOG, N, 0.9, 1.0, i - 1) == pytest.approx(0.9 * (1 + g * math.log(i)))
    assert O.beta_at(O.LINEAR, 1, 0.3, 9.0, 0) == 0.3


def test_thresholds_against_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    rng = np.random.default_rng(0)
    for _ in range(3000):
        beta = float(rng.choice([0.0, 0.02, 0.05, 0.9, 1.0, 3.7, 20.0, 30.0]) * rng.uniform(0.5, 1.5))
        dE = int(rng.integers(1, 40000))
        scale = int(rng.choice([1024, 4096]))
        T = O.accept_threshold(beta, dE, scale)
        x = mpmath.mpf(beta) * dE / scale
        exact = mpmath.ldexp(mpmath.exp(-x), 32)
        ref = min(2 ** 32 - 1, int(mpmath.floor(exact)))
        if abs(exact - mpmath.nint(exact)) < mpmath.mpf("1e-3") * max(1, exact) * 1e-9:
            continue   # exact value on an integer boundary: FP64 may round either way
        assert abs(T - ref) <= 1, (beta, dE, scale, T, ref)
        if exact > 1e6:
            assert abs(T - ref) / exact < 1e-12
    assert O.accept_threshold(0.0, 5, 1024) == 2 ** 32 - 1
    assert O.accept_threshold(1e6, 1, 4096) == 0


def test_thresholds_monotone():
    for beta in (0.05, 1.0, 20.0):
        T = [O.accept_threshold(beta, dE, 1024) for dE in range(1, 20000, 37)]
        assert all(a >= b for a, b in zip(T, T[1:]))
    T = [O.accept_threshold(O.beta_at(O.LINEAR, 50, 0.05, 20.0, t), 2260, 1024) for t in range(50)]
    assert all(a >= b for a, b in zip(T, T[1:]))
