"""Pins of the oracle's code tables against the algebra the paper fixes.

Sec. "The XZZX code": one generator type G_f = X Z Z X around each face
(Eq. stabilizer_generator), weight 4 in the bulk and lower on the boundary;
L_Z joins left and right, L_X top and bottom, L_Y = i L_Z L_X; the distance
equals the linear size.  The generators are read back from the oracle's own
syndrome map (the syndrome of a single-qubit X or Z), so a dropped corner, a
swapped X/Z or a wrong face fails the algebra below.
"""
import numpy as np
import pytest

import oracle as O
from codehelp import generators_from_syndromes
from gf2 import pauli_rows, rank, symplectic

DS = [3, 5, 7, 9, 11, 13]




@pytest.mark.parametrize("d", DS)
def test_counts_and_weights(d):
    nq, ns, cs = O.code_sizes(d)
    assert nq == d * d and ns == d * d - 1
    assert list(np.diff(cs)) == [(d * d - 1) // 4] * 4
    G = generators_from_syndromes(d)
    w = (G != 0).sum(1)
    assert sorted(set(w.tolist())) == [2, 4]
    assert (w == 4).sum() == (d - 1) ** 2 and (w == 2).sum() == 2 * (d - 1)


@pytest.mark.parametrize("d", DS)
def test_xzzx_pattern(d):
    """Each generator is X on TL and BR, Z on TR and BL (Eq. stabilizer_generator)."""
    faces = O.code_faces(d)
    G = generators_from_syndromes(d)
    expect = [2, 1, 1, 2]  # X, Z, Z, X on TL, TR, BL, BR
    for f in range(len(faces["a"])):
        a, b = faces["a"][f], faces["b"][f]
        corners = [(a, b), (a, b + 1), (a + 1, b), (a + 1, b + 1)]
        for k, (r, c) in enumerate(corners):
            inside = 0 <= r < d and 0 <= c < d
            assert faces["corners"][f][k] == (r * d + c if inside else -1)
            if inside:
                assert G[f, r * d + c] == expect[k]
        assert (G[f] != 0).sum() == sum(0 <= r < d and 0 <= c < d for r, c in corners)


@pytest.mark.parametrize("d", DS)
def test_commutation_rank_and_logicals(d):
    G = pauli_rows(generators_from_syndromes(d))
    assert not symplectic(G, G).any()              # all generators commute
    assert rank(G) == d * d - 1                    # independent
    LX, LZ = O.logicals(d)
    L = pauli_rows(np.stack([LX, LZ]))
    assert not symplectic(L, G).any()              # logicals commute with the group
    assert symplectic(L[:1], L[1:])[0, 0] == 1     # and anticommute with each other
    assert rank(np.vstack([G, L[:1]])) == d * d
    assert rank(np.vstack([G, L[1:]])) == d * d
    assert rank(np.vstack([G, L])) == d * d + 1
    # L_Z runs along the top row (left to right), L_X down the left column.
    assert set(np.nonzero(LZ)[0].tolist()) == set(range(d))
    assert set(np.nonzero(LX)[0].tolist()) == set(range(0, d * d, d))


@pytest.mark.parametrize("d", DS)
def test_colour_classes_disjoint(d):
    faces = O.code_faces(d)
    G = generators_from_syndromes(d)
    for c in range(4):
        idx = np.nonzero(faces["colour4"] == c)[0]
        support = (G[idx] != 0).astype(np.int64)
        assert (support.sum(0) <= 1).all()
    # stabilizer index order is colour-major
    assert (np.diff(faces["colour4"]) >= 0).all()


@pytest.mark.parametrize("d", [3, 5])
def test_distance_by_enumeration(d):
    """With equal weights (depolarizing, px:py:pz = 1:1:1) the minimum energy of
    the X and Z cosets of the empty syndrome is d times the weight: the code
    distance is the linear size (Sec. "The XZZX code").  The Y coset needs an X
    string and a Z string crossing on one qubit, 2d-1 qubits."""
    pxyz = O.noise_from_eta(0.06, 1.0, O.PAPER_ETA)
    W4, _ = O.make_noise(*pxyz, 1024)
    assert W4[1] == W4[2] == W4[3]
    E = O.bruteforce(d, pxyz, 1024, np.zeros(d * d, np.uint8))
    assert E[0] == 0
    assert list(E[1:]) == [d * W4[1], (2 * d - 1) * W4[1], d * W4[1]]


@pytest.mark.parametrize("d", [3, 5, 7])
def test_class_bits_of_logicals(d):
    LX, LZ = O.logicals(d)
    assert O.class_bits(d, LX) == 1          # X class
    assert O.class_bits(d, LZ) == 2          # Z class
    assert O.class_bits(d, LX ^ LZ) == 3     # Y class
    G = generators_from_syndromes(d)
    for f in range(G.shape[0]):
        assert O.class_bits(d, G[f]) == 0
