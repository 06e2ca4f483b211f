"""CPU checks of the C-ABI library: it loads, exports every entry point the
public header declares, validates its arguments, and its host tables (faces,
weights, acceptance thresholds) agree with the oracle's.  No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

import golden_data
import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def X():
    from paper_2509_17837_gb300 import build
    build.build()
    import paper_2509_17837_gb300 as X
    return X


def declared_functions():
    src = open(os.path.join(ROOT, "include", "xzzx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xzzx_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(X):
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2509_17837_gb300", "libxzzx.so"))
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_2509_17837_gb300._lib import SIGNATURES
    assert set(SIGNATURES) == set(names)


def test_ctypes_struct_layouts_match_the_library(X):
    """The binding's ctypes copies of the public structs have the sizes the
    library was compiled with (a field added on one side only fails here)."""
    from paper_2509_17837_gb300 import _lib as L
    mirrors = [L.Noise, L.CodeInfo, L.Segment, L.BatchCfg, L.BatchInfo, L.ServeCfg, L.Result, L.ServeStats]
    for which, cls in enumerate(mirrors):
        assert L.lib().xzzx_abi_struct_size(which) == ctypes.sizeof(cls), cls.__name__
    assert L.lib().xzzx_abi_struct_size(len(mirrors)) == 0
    assert L.lib().xzzx_abi_struct_size(-1) == 0


def test_argument_validation(X):
    from paper_2509_17837_gb300._lib import XZZX_EINVAL, XZZX_EUNSUPPORTED, XzzxError
    for d in (1, 2, 4, 33, 0, -3):
        with pytest.raises(XzzxError) as e:
            X.Code(d)
        assert e.value.status == XZZX_EINVAL
    with pytest.raises(XzzxError) as e:
        X.Code(5, layout=2)
    assert e.value.status == XZZX_EUNSUPPORTED
    for bad in ((0.0, 0.1, 0.1), (0.3, 0.2, 0.1), (-0.1, 0.1, 0.1)):
        with pytest.raises(XzzxError):
            X.make_noise(*bad)
    n = X.noise_from_eta(0.1, 10)
    with pytest.raises(XzzxError):
        X.Schedule(n, -1, 0.1, 1.0)
    with pytest.raises(XzzxError):
        X.Schedule(n, 10, float("nan"), 1.0)
    with pytest.raises(XzzxError):
        X.Schedule(n, 10, 0.0, 1.0, kind=X.PAPER_LOG)


@pytest.mark.parametrize("d", [3, 5, 11, 21, 31])
def test_faces_match_oracle(X, d):
    c = X.Code(d)
    a, b, corners = c.faces()
    of = O.code_faces(d)
    assert np.array_equal(a, of["a"]) and np.array_equal(b, of["b"])
    assert np.array_equal(corners, of["corners"])
    _, _, cs = O.code_sizes(d)
    assert c.colour_start == list(cs)
    assert c.words == (d * d + 31) // 32 and c.syn_words == (d * d - 1 + 31) // 32


@pytest.mark.parametrize("d", [3, 5, 11, 21, 31])
def test_planar_faces_match_oracle(X, d):
    """The library's planar tables (face sites, corner qubits, colour classes,
    index order) equal the oracle's pinned ones."""
    c = X.Code(d, layout=X.LAYOUT_PLANAR)
    a, b, corners = c.faces()
    cid = O.planar(d)
    of = O.code_faces(cid)
    assert np.array_equal(a, of["a"]) and np.array_equal(b, of["b"])
    assert np.array_equal(corners, of["corners"])
    nq, ns, cs = O.code_sizes(cid)
    assert c.colour_start == list(cs)
    assert c.n_qubits == nq and c.n_stab == ns
    assert c.words == (nq + 31) // 32 and c.syn_words == (ns + 31) // 32


@pytest.mark.parametrize("p,eta,conv,scale", [(0.10, 10, 0, 1024), (0.10, 100, 0, 1024), (0.22, 100, 0, 1024),
                                              (0.15, 1000, 0, 4096), (0.30, 1000, 0, 4096), (0.2, 1.0, 1, 1024),
                                              (0.12, 5, 1, 2048)])
def test_weights_match_oracle(X, p, eta, conv, scale):
    n = X.noise_from_eta(p, eta, conv, scale)
    pxyz = O.noise_from_eta(p, eta, conv)
    assert (n.px, n.py, n.pz) == pxyz
    W4, Wt = O.make_noise(*pxyz, scale)
    assert list(n.W) == list(W4) and [n.Wt_x, n.Wt_z] == list(Wt)


@pytest.mark.parametrize("p,eta,scale,wx,wy,wt", golden_data.weight_table())
def test_library_weights_equal_printed_table(X, p, eta, scale, wx, wy, wt):
    """xzzx_noise_from_eta gives the stored integer weights of Eqs. coeff_in_energy
    and coeff_in_distance."""
    n = X.noise_from_eta(p, eta, 0, scale)
    assert list(n.W) == [0, wx, wx, wy] and [n.Wt_x, n.Wt_z] == [wt, wt]


def reachable_positive_dE(W4):
    """Every energy change a generator can make (brute force): the bulk X Z Z X
    face, the rotated weight-2 faces and the planar three-body faces (X X Z
    and X Z Z)."""
    flip = [2, 1, 1, 2]
    out = set()
    for mask in (0xF, 0xC, 0x3, 0xA, 0x5, 0xB, 0x7):
        corners = [k for k in range(4) if (mask >> k) & 1]
        for labs in np.ndindex(*([4] * len(corners))):
            dE = sum(int(W4[l ^ flip[k]]) - int(W4[l]) for k, l in zip(corners, labs))
            if dE > 0:
                out.add(dE)
    return sorted(out)


@pytest.mark.parametrize("kind,N,b0,b1", [(0, 1000, 0.05, 20.0), (0, 200, 0.1, 10.0), (1, 100, 0.9, 1.0),
                                          (0, 1, 0.3, 7.0), (0, 37, 0.0, 0.0), (0, 5, 1e6, 1e6)])
def test_thresholds_match_oracle(X, kind, N, b0, b1):
    n = X.noise_from_eta(0.13, 100)
    s = X.Schedule(n, N, b0, b1, kind=kind)
    dE, T = s.table()
    assert list(dE) == reachable_positive_dE(list(n.W))
    for t in range(N):
        beta = O.beta_at(kind, N, b0, b1, t)
        ref = [O.accept_threshold(beta, int(e), n.scale) for e in dE]
        assert list(T[t]) == ref, t
