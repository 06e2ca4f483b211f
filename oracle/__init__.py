"""ctypes wrapper of the oracle (test infrastructure only).

The oracle is a plain single-threaded C++ restatement of the XZZX
simulated-annealing decoder of arXiv:2509.17837 (see ``oracle.cpp``).  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
import this package; the product path never does.

Configurations are numpy ``uint8`` arrays with one two-bit Pauli per qubit
(I=0, Z=1, X=2, Y=3); syndromes are ``uint8`` arrays with one bit per
stabilizer in stabilizer-index order.

Every function takes a code id: the distance d for the rotated layout, or
``planar(d)`` for the paper's planar layout.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

LINEAR, PAPER_LOG = 0, 1
INIT_GREEDY, INIT_GREEDY_RANDOM, INIT_BOUNDARY = 0, 1, 2
ORDER_COLOUR, ORDER_RANDOM_SITE = 0, 1
EMIN_PER_PHASE, EMIN_PER_ATTEMPT = 0, 1
Y_OVER_XZ_ETA, PAPER_ETA = 0, 1
PLANAR_ID = 1000


def planar(d):
    """Code id of the planar layout of distance d."""
    return d + PLANAR_ID


def distance(code_id):
    return code_id % PLANAR_ID


def _nq(d):
    return code_sizes(d)[0]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        i32, u64, dbl = C.c_int, C.c_uint64, C.c_double
        p = C.c_void_p
        L.orc_philox.argtypes = [u64, p, p]
        L.orc_code_sizes.argtypes = [i32, p, p, p]
        L.orc_code_faces.argtypes = [i32, p, p, p, p, p]
        L.orc_logicals.argtypes = [i32, p, p]
        L.orc_make_noise.argtypes = [dbl, dbl, dbl, C.c_int32, p, p]
        L.orc_noise_from_eta.argtypes = [dbl, dbl, i32, p]
        L.orc_sample.argtypes = [i32, dbl, dbl, dbl, u64, u64, i32, p, p]
        L.orc_syndrome.argtypes = [i32, p, p]
        L.orc_class_bits.argtypes = [i32, p]
        L.orc_boundary_distance.argtypes = [i32, dbl, dbl, dbl, C.c_int32, p]
        L.orc_greedy.argtypes = [i32, dbl, dbl, dbl, C.c_int32, u64, u64, i32, i32, p, p, p]
        L.orc_walk_internal.argtypes = [i32, i32, i32, p]
        L.orc_walk_boundary.argtypes = [i32, dbl, dbl, dbl, C.c_int32, i32, p]
        L.orc_beta_at.argtypes = [i32, i32, dbl, dbl, i32]
        L.orc_beta_at.restype = dbl
        L.orc_accept_threshold.argtypes = [dbl, C.c_int32, C.c_int32]
        L.orc_accept_threshold.restype = C.c_uint32
        L.orc_anneal_chain.argtypes = [i32, dbl, dbl, dbl, C.c_int32, i32, i32, dbl, dbl, u64, u64,
                                       p, p, p, p, p, p]
        L.orc_anneal_chain_variant.argtypes = [i32, dbl, dbl, dbl, C.c_int32, i32, i32, dbl, dbl, u64, u64, p,
                                               i32, i32, p, p, p, p, p]
        L.orc_decode.argtypes = [i32, dbl, dbl, dbl, C.c_int32, i32, i32, dbl, dbl, u64, u64, i32, i32,
                                 i32, p, p, p, p, p, p, p, p, p]
        L.orc_bruteforce.argtypes = [i32, dbl, dbl, dbl, C.c_int32, p, p]
        L.orc_coset_energies.argtypes = [i32, dbl, dbl, dbl, C.c_int32, p, p]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def philox(key, ctr):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox(key, _ptr(ctr), _ptr(out))
    return out


def code_sizes(d):
    nq, ns = C.c_int(), C.c_int()
    cs = np.zeros(5, np.int32)
    _check(lib().orc_code_sizes(d, C.byref(nq), C.byref(ns), _ptr(cs)), "code_sizes")
    return nq.value, ns.value, cs


def code_faces(d):
    _, ns, _ = code_sizes(d)
    a, b, c4, c2 = (np.zeros(ns, np.int32) for _ in range(4))
    corners = np.zeros((ns, 4), np.int32)
    _check(lib().orc_code_faces(d, _ptr(a), _ptr(b), _ptr(c4), _ptr(c2), _ptr(corners)), "code_faces")
    return dict(a=a, b=b, colour4=c4, colour2=c2, corners=corners)


def logicals(d):
    nq = _nq(d)
    LX, LZ = np.zeros(nq, np.uint8), np.zeros(nq, np.uint8)
    _check(lib().orc_logicals(d, _ptr(LX), _ptr(LZ)), "logicals")
    return LX, LZ


def noise_from_eta(p, eta, convention=Y_OVER_XZ_ETA):
    out = np.zeros(3, np.float64)
    _check(lib().orc_noise_from_eta(p, eta, convention, _ptr(out)), "noise_from_eta")
    return tuple(float(x) for x in out)


def make_noise(px, py, pz, scale):
    W4 = np.zeros(4, np.int32)
    Wt = np.zeros(2, np.int32)
    _check(lib().orc_make_noise(px, py, pz, scale, _ptr(W4), _ptr(Wt)), "make_noise")
    return W4, Wt


def sample(d, pxyz, seed, shot0, n_shots):
    nq, ns, _ = code_sizes(d)
    err = np.zeros((n_shots, nq), np.uint8)
    syn = np.zeros((n_shots, ns), np.uint8)
    _check(lib().orc_sample(d, *pxyz, seed, shot0, n_shots, _ptr(err), _ptr(syn)), "sample")
    return err, syn


def syndrome(d, cfg):
    _, ns, _ = code_sizes(d)
    cfg = np.ascontiguousarray(cfg, np.uint8)
    out = np.zeros(ns, np.uint8)
    _check(lib().orc_syndrome(d, _ptr(cfg), _ptr(out)), "syndrome")
    return out


def class_bits(d, cfg):
    cfg = np.ascontiguousarray(cfg, np.uint8)
    r = lib().orc_class_bits(d, _ptr(cfg))
    if r < 0:
        raise RuntimeError("class_bits")
    return r


def boundary_distance(d, pxyz, scale):
    _, ns, _ = code_sizes(d)
    out = np.zeros(ns, np.int64)
    _check(lib().orc_boundary_distance(d, *pxyz, scale, _ptr(out)), "boundary_distance")
    return out


def greedy(d, pxyz, scale, seed, shot, restart, randomised, syn):
    syn = np.ascontiguousarray(syn, np.uint8)
    R = np.zeros(_nq(d), np.uint8)
    w = C.c_int64()
    _check(lib().orc_greedy(d, *pxyz, scale, seed, shot, restart, randomised, _ptr(syn), _ptr(R),
                            C.byref(w)), "greedy")
    return R, w.value


def walk_internal(d, u, v):
    R = np.zeros(_nq(d), np.uint8)
    rc = lib().orc_walk_internal(d, u, v, _ptr(R))
    return (R if rc == 0 else None)


def walk_boundary(d, pxyz, scale, u):
    R = np.zeros(_nq(d), np.uint8)
    rc = lib().orc_walk_boundary(d, *pxyz, scale, u, _ptr(R))
    return (R if rc == 0 else None)


def beta_at(kind, n_sweeps, beta0, beta1, t):
    return lib().orc_beta_at(kind, n_sweeps, beta0, beta1, t)


def accept_threshold(beta, dE, scale):
    return int(lib().orc_accept_threshold(beta, dE, scale))


def anneal_chain(d, pxyz, scale, kind, n_sweeps, beta0, beta1, seed, chain, init, trace=False):
    init = np.ascontiguousarray(init, np.uint8)
    nq = _nq(d)
    best, fin = np.zeros(nq, np.uint8), np.zeros(nq, np.uint8)
    bE, fE = C.c_int32(), C.c_int32()
    tr = np.zeros(max(n_sweeps, 1), np.int32) if trace else None
    _check(lib().orc_anneal_chain(d, *pxyz, scale, kind, n_sweeps, beta0, beta1, seed, chain, _ptr(init),
                                  _ptr(best), C.byref(bE), _ptr(fin), C.byref(fE), _ptr(tr)), "anneal_chain")
    out = dict(best=best, best_E=bE.value, final=fin, final_E=fE.value)
    if trace:
        out["trace_E"] = tr[:n_sweeps]
    return out


def decode(d, pxyz, scale, kind, n_sweeps, beta0, beta1, seed, shot0, restarts, syn, err=None,
           randomised=1, want_chains=False):
    syn = np.ascontiguousarray(syn, np.uint8)
    n = syn.shape[0]
    nq = _nq(d)
    cls = np.zeros(n, np.uint8)
    E4 = np.zeros((n, 4), np.int32)
    rec = np.zeros((n, nq), np.uint8)
    best = np.zeros((n, nq), np.uint8)
    fail = np.zeros(n, np.uint8) if err is not None else None
    chainE = np.zeros((n, 4 * restarts), np.int32) if want_chains else None
    qb = np.zeros((n, restarts), np.uint8) if want_chains else None
    if err is not None:
        err = np.ascontiguousarray(err, np.uint8)
    _check(lib().orc_decode(d, *pxyz, scale, kind, n_sweeps, beta0, beta1, seed, shot0, n, restarts,
                            randomised, _ptr(syn), _ptr(err), _ptr(cls), _ptr(E4), _ptr(rec), _ptr(best),
                            _ptr(fail), _ptr(chainE), _ptr(qb)), "decode")
    out = dict(cls=cls, E4=E4, recovery=rec, best_cfg=best)
    if fail is not None:
        out["fail"] = fail
    if want_chains:
        out["chain_E"] = chainE
        out["q_bits"] = qb
    return out


def bruteforce(d, pxyz, scale, R):
    R = np.ascontiguousarray(R, np.uint8)
    out = np.zeros(4, np.int32)
    _check(lib().orc_bruteforce(d, *pxyz, scale, _ptr(R), _ptr(out)), "bruteforce")
    return out


def coset_energies(d, pxyz, scale, start):
    start = np.ascontiguousarray(start, np.uint8)
    m = code_sizes(d)[1]
    out = np.zeros(1 << m, np.int32)
    _check(lib().orc_coset_energies(d, *pxyz, scale, _ptr(start), _ptr(out)), "coset_energies")
    return out


def anneal_chain_variant(d, pxyz, scale, kind, n_sweeps, beta0, beta1, seed, chain, init, order, emin,
                         trace=False):
    init = np.ascontiguousarray(init, np.uint8)
    nq = _nq(d)
    best, fin = np.zeros(nq, np.uint8), np.zeros(nq, np.uint8)
    bE, fE = C.c_int32(), C.c_int32()
    tr = np.zeros(max(n_sweeps, 1), np.int32) if trace else None
    _check(lib().orc_anneal_chain_variant(d, *pxyz, scale, kind, n_sweeps, beta0, beta1, seed, chain, _ptr(init),
                                          order, emin, _ptr(best), C.byref(bE), _ptr(fin), C.byref(fE), _ptr(tr)),
           "anneal_chain_variant")
    out = dict(best=best, best_E=bE.value, final=fin, final_E=fE.value)
    if trace:
        out["trace_E"] = tr[:n_sweeps]
    return out
