"""Pins of the oracle's planar layout: the paper's own lattice (Sec. "The XZZX
code"): d^2 + (d-1)^2 data qubits, 2d(d-1) generators, four-body in the bulk
and three-body on the boundary, L_Z joining left and right, L_X top and bottom.

The generators are read back from the oracle's syndrome map, so the algebra
below checks what the oracle computes, not what it was told.  The generic
pins of the other oracle test files (shortest paths, greedy >= MWPM, chain
invariants, detailed balance, single-error correction) also run on planar
code ids; this file adds what is specific to the planar geometry: corner
positions, counts, the colour classes and draw coordinates, the paper's closed
forms for w(u, b) and w_int (Eqs. distance_u_boundary, distance_u_v_internal),
the distance, and exact coset minima on the d = 3 planar workload.
"""
import math

import numpy as np
import pytest

import oracle as O
from codehelp import generators_from_syndromes
from gf2 import pauli_rows, rank, symplectic

DS = [3, 5, 7, 9]


def qubit_site_index(d, r, c):
    """Row-major index over the qubit sites (r + c even) of the (2d-1)^2 grid."""
    g = 2 * d - 1
    if not (0 <= r < g and 0 <= c < g) or (r + c) % 2:
        return -1
    sites = [(i, j) for i in range(g) for j in range(g) if (i + j) % 2 == 0]
    return sites.index((r, c))


@pytest.mark.parametrize("d", DS)
def test_counts_and_weights(d):
    nq, ns, cs = O.code_sizes(O.planar(d))
    assert nq == d * d + (d - 1) ** 2 and ns == 2 * d * (d - 1)
    G = generators_from_syndromes(O.planar(d))
    w = (G != 0).sum(1)
    assert (w == 4).sum() == 2 * (d - 1) * (d - 2) and (w == 3).sum() == 4 * (d - 1)
    assert int(cs[4]) == ns and (np.diff(cs) > 0).all()


@pytest.mark.parametrize("d", [3, 5])
def test_xzzx_pattern_and_qubit_index(d):
    """G_f = X_left Z_up Z_down X_right (Eq. stabilizer_generator) around every
    face (i, j), i + j odd; qubit (r, c) has the row-major site index."""
    cid = O.planar(d)
    faces = O.code_faces(cid)
    G = generators_from_syndromes(cid)
    expect = [2, 1, 1, 2]  # X left, Z up, Z down, X right
    for f in range(len(faces["a"])):
        i, j = int(faces["a"][f]), int(faces["b"][f])
        assert (i + j) % 2 == 1
        sites = [(i, j - 1), (i - 1, j), (i + 1, j), (i, j + 1)]
        n_in = 0
        for k, (r, c) in enumerate(sites):
            q = qubit_site_index(d, r, c)
            assert faces["corners"][f][k] == q
            if q >= 0:
                n_in += 1
                assert G[f, q] == expect[k]
        assert (G[f] != 0).sum() == n_in


@pytest.mark.parametrize("d", DS)
def test_commutation_rank_and_logicals(d):
    cid = O.planar(d)
    nq, ns, _ = O.code_sizes(cid)
    G = pauli_rows(generators_from_syndromes(cid))
    assert not symplectic(G, G).any()
    assert rank(G) == ns == nq - 1                  # one logical qubit
    LX, LZ = O.logicals(cid)
    L = pauli_rows(np.stack([LX, LZ]))
    assert not symplectic(L, G).any()
    assert symplectic(L[:1], L[1:])[0, 0] == 1
    assert rank(np.vstack([G, L[:1]])) == nq
    assert rank(np.vstack([G, L[1:]])) == nq
    assert rank(np.vstack([G, L])) == nq + 1
    g = 2 * d - 1
    row0 = {qubit_site_index(d, 0, c) for c in range(0, g, 2)}
    col0 = {qubit_site_index(d, r, 0) for r in range(0, g, 2)}
    assert set(np.nonzero(LZ)[0].tolist()) == row0 and set(LZ[list(row0)].tolist()) == {1}
    assert set(np.nonzero(LX)[0].tolist()) == col0 and set(LX[list(col0)].tolist()) == {2}


@pytest.mark.parametrize("d", [3, 5, 7, 11, 31])
def test_colours_and_draw_coordinates(d):
    """Same-colour generators have disjoint supports; the index order is
    (colour, j>>2, i>>1), and (i>>1, j>>2) names each face of a colour once, so
    four faces with consecutive i>>1 share one draw block."""
    cid = O.planar(d)
    faces = O.code_faces(cid)
    a, b, c4 = faces["a"], faces["b"], faces["colour4"]
    key = [(int(c4[f]), int(b[f]) >> 2, int(a[f]) >> 1) for f in range(len(a))]
    assert key == sorted(key) and len(set(key)) == len(key)
    corners = faces["corners"]
    for c in range(4):
        used = [q for f in np.nonzero(c4 == c)[0] for q in corners[f] if q >= 0]
        assert len(used) == len(set(used))
    # decoding-graph colour: faces on even rows (left/right boundaries) vs odd rows
    assert (faces["colour2"] == (a & 1)).all()


@pytest.mark.parametrize("d", [3, 5, 9, 15])
@pytest.mark.parametrize("pxyz", [(0.02, 0.05, 0.08), (0.01, 0.1, 0.01)])
def test_closed_forms_of_the_paper(d, pxyz):
    """On the planar lattice the oracle's graph distances are the paper's closed
    forms: w(u, b) = Wt_z min(dist_L, dist_R) on the faces meeting the left
    and right boundaries and Wt_x min(dist_B, dist_T) on the others
    (Eq. distance_u_boundary), and w_int is the weighted Manhattan distance
    (Eq. distance_u_v_internal), here checked through the internal walk."""
    cid = O.planar(d)
    _, Wt = O.make_noise(*pxyz, 1024)
    wb = O.boundary_distance(cid, pxyz, 1024)
    faces = O.code_faces(cid)
    for f in range(len(wb)):
        i, j = int(faces["a"][f]), int(faces["b"][f])
        if i % 2 == 0:
            ux = (j + 1) // 2                       # column of the vertex, 1..d-1
            assert wb[f] == Wt[1] * min(ux, d - ux)
        else:
            uy = (i + 1) // 2
            assert wb[f] == Wt[0] * min(uy, d - uy)
    rng = np.random.default_rng(d)
    ns = len(wb)
    for _ in range(200):
        u, v = (int(x) for x in rng.choice(ns, 2, replace=False))
        if faces["colour2"][u] != faces["colour2"][v]:
            continue
        P = O.walk_internal(cid, u, v)
        dj = abs(int(faces["b"][u]) - int(faces["b"][v])) // 2
        di = abs(int(faces["a"][u]) - int(faces["a"][v])) // 2
        assert P is not None
        assert (P & 1).sum() == dj and ((P >> 1) & 1).sum() == di      # Z steps, X steps
        syn = np.zeros(ns, np.uint8)
        syn[[u, v]] = 1
        assert np.array_equal(O.syndrome(cid, P), syn)


def test_distance_by_enumeration():
    """Equal weights: the X and Z cosets of the trivial syndrome cost d qubits,
    the Y coset 2d - 1 (an X string and a Z string crossing on one qubit)."""
    d = 3
    pxyz = O.noise_from_eta(0.06, 1.0, O.PAPER_ETA)
    W4, _ = O.make_noise(*pxyz, 1024)
    nq = O.code_sizes(O.planar(d))[0]
    E = O.bruteforce(O.planar(d), pxyz, 1024, np.zeros(nq, np.uint8))
    assert E[0] == 0
    assert list(E[1:]) == [d * W4[1], (2 * d - 1) * W4[1], d * W4[1]]


def test_sa_reaches_exact_coset_minima_planar_d3():
    """The d = 3 planar workload (p = 0.10, 1:10:1, 8 restarts, 200 sweeps):
    SA never undercuts the exact coset minima and reaches the global minimum on
    at least 99.9% of 400 shots."""
    cid, shots, scale = O.planar(3), 400, 1024
    pxyz = O.noise_from_eta(0.10, 10, O.PAPER_ETA)
    err, syn = O.sample(cid, pxyz, 0xB3, 0, shots)
    out = O.decode(cid, pxyz, scale, O.LINEAR, 200, 0.1, 10.0, 0xB3, 0, 8, syn, err)
    hits = 0
    for s in range(shots):
        R1, _ = O.greedy(cid, pxyz, scale, 0xB3, s, 0, 1, syn[s])
        bf = O.bruteforce(cid, pxyz, scale, R1)
        assert (out["E4"][s] >= bf).all()
        hits += out["E4"][s].min() == bf.min()
    assert hits >= math.ceil(0.999 * shots)


@pytest.mark.parametrize("order,emin", [(1, 0), (1, 1), (0, 1)])
def test_variants_keep_syndrome_and_coset(order, emin):
    cid = O.planar(5)
    pxyz = O.noise_from_eta(0.15, 5, O.PAPER_ETA)
    W4, _ = O.make_noise(*pxyz, 1024)
    err, syn = O.sample(cid, pxyz, 4, 0, 3)
    for s in range(3):
        R, _ = O.greedy(cid, pxyz, 1024, 4, s, 0, 1, syn[s])
        out = O.anneal_chain_variant(cid, pxyz, 1024, O.PAPER_LOG, 30, 0.9, 1.0, 4, s, R, order, emin)
        for key in ("best", "final"):
            assert np.array_equal(O.syndrome(cid, out[key]), syn[s])
            assert O.class_bits(cid, out[key] ^ R) == 0
            assert out[key + "_E"] == int(np.asarray(W4, np.int64)[out[key]].sum())
