"""Pins of the oracle's greedy matching (Algs. 5 and 6) and its paths.

The decoding graphs of Sec. "Principles of error detection and correction" are
rebuilt here from the oracle's syndrome map (each X or Z component of a qubit
is an edge between the faces it flags; a single flagged face makes a boundary
edge) and searched with networkx, independent of the oracle's own formulas:

* w(u, b) and w(u, v) = min(w_int, w_bnd) (Eqs. distance_u_v_def_new,
  distance_u_boundary) equal the graph shortest paths;
* every path the oracle draws has the syndrome of its end points and the
  weight of a shortest path;
* greedy recoveries reproduce the syndrome and never beat the minimum-weight
  perfect matching (Sec. "The MWPM decoder versus our SA decoder");
* the randomised tie-breaking matches the distribution of Alg. 6 taken
  literally (uniform picks among the remaining minimum-weight pairs),
  enumerated exactly on small defect sets.
"""
import itertools
import math
from fractions import Fraction

import networkx as nx
import numpy as np
import pytest

import oracle as O
from inputs import random_syndromes

B = "boundary"


def decoding_graph(d, Wt):
    """networkx graph of both colours plus one boundary node; edge attr q, comp."""
    nq = O.code_sizes(d)[0]
    G = nx.Graph()
    _, ns, _ = O.code_sizes(d)
    G.add_nodes_from(range(ns))
    G.add_node(B)
    for q in range(nq):
        for lab, w in ((2, Wt[0]), (1, Wt[1])):   # X component weighs Wt_x, Z component Wt_z
            cfg = np.zeros(nq, np.uint8)
            cfg[q] = lab
            flagged = np.nonzero(O.syndrome(d, cfg))[0].tolist()
            assert len(flagged) in (1, 2)
            u, v = (flagged + [B])[:2]
            if G.has_edge(u, v):
                G[u][v]["weight"] = min(G[u][v]["weight"], w)
            else:
                G.add_edge(u, v, weight=int(w))
    return G


def cfg_weight(cfg, Wt):
    x = ((cfg >> 1) & 1).sum()
    z = (cfg & 1).sum()
    return int(x) * int(Wt[0]) + int(z) * int(Wt[1])


NOISES = {
    "equal": (O.noise_from_eta(0.15, 100), 1024),
    "unequal": ((0.02, 0.05, 0.08), 1024),   # Wt_x != Wt_z
}


@pytest.mark.parametrize("d", [3, 5, 11, 25, O.planar(3), O.planar(5), O.planar(11)])
@pytest.mark.parametrize("noise", ["equal", "unequal"])
def test_boundary_distance_is_shortest_path(d, noise):
    pxyz, scale = NOISES[noise]
    _, Wt = O.make_noise(*pxyz, scale)
    G = decoding_graph(d, Wt)
    dist = nx.single_source_dijkstra_path_length(G, B)
    wb = O.boundary_distance(d, pxyz, scale)
    assert [dist[f] for f in range(len(wb))] == wb.tolist()


@pytest.mark.parametrize("d", [3, 5, 7, 11, O.planar(3), O.planar(5), O.planar(7)])
@pytest.mark.parametrize("noise", ["equal", "unequal"])
def test_pair_weight_and_paths(d, noise):
    pxyz, scale = NOISES[noise]
    _, Wt = O.make_noise(*pxyz, scale)
    G = decoding_graph(d, Wt)
    Gint = G.copy()
    Gint.remove_node(B)
    faces = O.code_faces(d)
    ns = len(faces["a"])
    full = dict(nx.all_pairs_dijkstra_path_length(G))
    inner = dict(nx.all_pairs_dijkstra_path_length(Gint))
    wb = O.boundary_distance(d, pxyz, scale)
    rng = np.random.default_rng(d)
    pairs = [(u, v) for u in range(ns) for v in range(u + 1, ns) if faces["colour2"][u] == faces["colour2"][v]]
    if len(pairs) > 600:
        pairs = [pairs[i] for i in rng.choice(len(pairs), 600, replace=False)]
    for u, v in pairs:
        syn = np.zeros(ns, np.uint8)
        syn[[u, v]] = 1
        R, w = O.greedy(d, pxyz, scale, 1, 0, 0, 1, syn)
        assert w == full[u][v]                                   # w(u,v) = min(w_int, w_bnd)
        assert np.array_equal(O.syndrome(d, R), syn)
        assert cfg_weight(R, Wt) == w
        P = O.walk_internal(d, u, v)
        assert P is not None and np.array_equal(O.syndrome(d, P), syn)
        assert cfg_weight(P, Wt) == inner[u][v]                  # a shortest internal path
    for u in range(ns):
        P = O.walk_boundary(d, pxyz, scale, u)
        one = np.zeros(ns, np.uint8)
        one[u] = 1
        assert P is not None and np.array_equal(O.syndrome(d, P), one)
        assert cfg_weight(P, Wt) == wb[u]


@pytest.mark.parametrize("d", [25, 31])
def test_internal_walk_large_lattices(d):
    faces = O.code_faces(d)
    ns = len(faces["a"])
    rng = np.random.default_rng(7)
    _, Wt = O.make_noise(*NOISES["equal"][0], 1024)
    for _ in range(300):
        u, v = rng.choice(ns, 2, replace=False)
        if faces["colour2"][u] != faces["colour2"][v]:
            continue
        P = O.walk_internal(d, int(u), int(v))
        assert P is not None
        ds = abs((faces["a"][u] + faces["b"][u]) - (faces["a"][v] + faces["b"][v])) // 2
        dd = abs((faces["a"][u] - faces["b"][u]) - (faces["a"][v] - faces["b"][v])) // 2
        assert (P & 1).sum() == ds and ((P >> 1) & 1).sum() == dd


@pytest.mark.parametrize("d,density", [(3, 0.3), (5, 0.25), (7, 0.2), (11, 0.15), (31, 0.1), (O.planar(3), 0.3),
                                       (O.planar(7), 0.2), (O.planar(21), 0.1)])
def test_greedy_reproduces_syndrome(d, density):
    _, ns, _ = O.code_sizes(d)
    pxyz, scale = NOISES["equal"]
    syns = random_syndromes(ns, 30 if ns < 900 else 6, density, seed=d)
    for s, syn in enumerate(syns):
        for r in range(3):
            for randomised in (0, 1):
                R, w = O.greedy(d, pxyz, scale, 5, s, r, randomised, syn)
                assert np.array_equal(O.syndrome(d, R), syn)


def mwpm_weight(G, defects):
    """Minimum-weight perfect matching over defects (+ b if odd) with w = graph distance."""
    dist = {u: nx.single_source_dijkstra_path_length(G, u) for u in defects}
    nodes = list(defects) + ([B] if len(defects) % 2 else [])
    K = nx.Graph()
    for a, b in itertools.combinations(nodes, 2):
        w = dist[a][b] if b != B else dist[a][B]
        K.add_edge(a, b, weight=w)
    if not nodes:
        return 0
    M = nx.min_weight_matching(K)
    assert 2 * len(M) == len(nodes)
    return sum(K[a][b]["weight"] for a, b in M)


@pytest.mark.parametrize("d", [5, 7, 9, O.planar(5), O.planar(7)])
@pytest.mark.parametrize("noise", ["equal", "unequal"])
def test_greedy_not_below_mwpm(d, noise):
    pxyz, scale = NOISES[noise]
    _, Wt = O.make_noise(*pxyz, scale)
    G = decoding_graph(d, Wt)
    faces = O.code_faces(d)
    _, ns, _ = O.code_sizes(d)
    syns = random_syndromes(ns, 25, 0.2, seed=100 + d)
    for s, syn in enumerate(syns):
        R, w = O.greedy(d, pxyz, scale, 3, s, 0, 1, syn)
        opt = 0
        for c in (0, 1):
            D = [f for f in range(ns) if syn[f] and faces["colour2"][f] == c]
            opt += mwpm_weight(G, D)
        assert w >= opt
        assert cfg_weight(R, Wt) <= w          # XOR of paths can only cancel edges


def alg6_distribution(defects, weight):
    """Exact outcome distribution of Alg. 6 taken literally: repeatedly pick a
    pair uniformly among the remaining pairs of minimum weight."""
    nodes = list(defects) + ([B] if len(defects) % 2 else [])
    out = {}

    def rec(free, chosen, prob):
        pairs = [(a, b) for a, b in itertools.combinations(sorted(free, key=str), 2)]
        if not pairs:
            key = frozenset(chosen)
            out[key] = out.get(key, 0) + prob
            return
        wmin = min(weight(a, b) for a, b in pairs)
        kmin = [p for p in pairs if weight(*p) == wmin]
        for a, b in kmin:
            rec(free - {a, b}, chosen + [frozenset((a, b))], prob / len(kmin))

    rec(frozenset(nodes), [], Fraction(1))
    return out


def matching_cfg(d, pxyz, scale, matching, full, inner):
    nq = O.code_sizes(d)[0]
    R = np.zeros(nq, np.uint8)
    for pair in matching:
        a, b = sorted(pair, key=str)
        if b == B:
            R ^= O.walk_boundary(d, pxyz, scale, a)
        elif inner[a][b] <= full[a][B] + full[b][B]:
            R ^= O.walk_internal(d, a, b)
        else:
            R ^= O.walk_boundary(d, pxyz, scale, a) ^ O.walk_boundary(d, pxyz, scale, b)
    return R.tobytes()


@pytest.mark.parametrize("case", range(6))
def test_tie_breaking_matches_alg6(case):
    d = 7
    pxyz, scale = NOISES["equal"]
    _, Wt = O.make_noise(*pxyz, scale)
    G = decoding_graph(d, Wt)
    Gint = G.copy()
    Gint.remove_node(B)
    faces = O.code_faces(d)
    ns = len(faces["a"])
    rng = np.random.default_rng(1000 + case)
    col0 = [f for f in range(ns) if faces["colour2"][f] == 0]
    defects = sorted(rng.choice(col0, int(rng.integers(3, 7)), replace=False).tolist())
    full = {u: nx.single_source_dijkstra_path_length(G, u) for u in defects}
    inner = {u: nx.single_source_dijkstra_path_length(Gint, u) for u in defects}

    def weight(a, b):
        if B in (a, b):
            return full[a if b == B else b][B]
        return full[a][b]

    exact = alg6_distribution(defects, weight)
    by_cfg = {}
    for m, pr in exact.items():
        k = matching_cfg(d, pxyz, scale, m, full, inner)
        by_cfg[k] = by_cfg.get(k, 0) + pr
    syn = np.zeros(ns, np.uint8)
    syn[defects] = 1
    n = 1500
    counts = {}
    for r in range(n):
        R, _ = O.greedy(d, pxyz, scale, 77, case, r, 1, syn)
        counts[R.tobytes()] = counts.get(R.tobytes(), 0) + 1
    assert set(counts) <= set(by_cfg), "greedy produced a matching Alg. 6 cannot produce"
    chi2 = 0.0
    for k, pr in by_cfg.items():
        e = n * float(pr)
        chi2 += (counts.get(k, 0) - e) ** 2 / e
    dof = max(len(by_cfg) - 1, 1)
    assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10
    # Alg. 5 (no randomisation) is deterministic
    R0 = {O.greedy(d, pxyz, scale, s, case, r, 0, syn)[0].tobytes() for s in (1, 2) for r in (0, 5)}
    assert len(R0) == 1 and next(iter(R0)) in by_cfg
