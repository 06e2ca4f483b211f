"""Run the oracle over many shots on every host core.

Workers are plain module-level functions so that a ``spawn`` pool can import
them; each worker process loads its own copy of the single-threaded oracle.
The pool is always started with the ``spawn`` method, so it is safe to use
after CUDA has been initialised in the parent.
"""
import multiprocessing as mp
import os

import numpy as np


def n_workers(n_tasks):
    return max(1, min(n_tasks, os.cpu_count() or 1))


def run(fn, tasks):
    """fn over tasks on a spawn pool (in order); serial when there is one core."""
    tasks = list(tasks)
    if n_workers(len(tasks)) == 1:
        return [fn(t) for t in tasks]
    with mp.get_context("spawn").Pool(n_workers(len(tasks))) as pool:
        return pool.map(fn, tasks, chunksize=1)


def chunks(lo, hi, n):
    """Split [lo, hi) into at most n contiguous (start, stop) ranges."""
    n = max(1, min(n, hi - lo))
    edges = np.linspace(lo, hi, n + 1).round().astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


def bruteforce_vs_sa(task):
    """Decode shots [s0, s1) with the oracle and compare each shot's coset
    energies with the exact coset minima found by enumerating the stabilizer
    group.  Returns per-shot (E4 from SA, exact E4, cls from SA, SA failure
    flag, failure flag of the exact minimum-energy decision, failure flag of
    the decision from the initial configurations alone (0 sweeps))."""
    import oracle as O
    c, s0, s1 = task
    pxyz = O.noise_from_eta(c["p"], c["eta"])
    err, syn = O.sample(c["d"], pxyz, c["seed"], s0, s1 - s0)
    out = O.decode(c["d"], pxyz, c["scale"], O.LINEAR, c["sweeps"], c["b0"], c["b1"], c["seed"], s0,
                   c["restarts"], syn, err)
    none = O.decode(c["d"], pxyz, c["scale"], O.LINEAR, 0, c["b0"], c["b1"], c["seed"], s0, c["restarts"], syn, err)
    LX, LZ = O.logicals(c["d"])
    Ls = [0 * LX, LX, LX ^ LZ, LZ]
    exact = np.zeros((s1 - s0, 4), np.int32)
    med_fail = np.zeros(s1 - s0, np.uint8)
    for i in range(s1 - s0):
        R1, _ = O.greedy(c["d"], pxyz, c["scale"], c["seed"], s0 + i, 0, 1, syn[i])
        exact[i] = O.bruteforce(c["d"], pxyz, c["scale"], R1)
        med_fail[i] = O.class_bits(c["d"], err[i] ^ R1 ^ Ls[int(np.argmin(exact[i]))]) != 0
    return out["E4"], exact, out["cls"], out["fail"], med_fail, none["fail"]


def decode_shots(task):
    """Oracle decode of the listed shot ids (each decoded alone; results do
    not depend on the batch).  task = (code_id, (px, py, pz), scale, kind,
    n_sweeps, beta0, beta1, seed, restarts, randomised, shot_ids).  Returns the
    per-shot dict of arrays, shots in the listed order."""
    import oracle as O
    d, pxyz, scale, kind, n_sweeps, b0, b1, seed, restarts, randomised, shots = task
    keys = ("cls", "E4", "recovery", "best_cfg", "fail", "chain_E", "q_bits")
    acc = {k: [] for k in keys}
    for s in shots:
        err, syn = O.sample(d, pxyz, seed, int(s), 1)
        out = O.decode(d, pxyz, scale, kind, n_sweeps, b0, b1, seed, int(s), restarts, syn, err,
                       randomised=randomised, want_chains=True)
        for k in keys:
            acc[k].append(out[k][0])
    return {k: np.array(v) for k, v in acc.items()}


def anneal_one_chain(task):
    """The oracle's greedy reference R_i of one (shot, restart), its class
    bits, and the best energy of chain (shot, restart, coset P) annealed from
    R_i L_P.  task = (code_id, (px, py, pz), scale, n_sweeps, beta0, beta1,
    seed, restarts, shot, restart, P); linear schedule, Alg. 6 references."""
    import oracle as O
    d, pxyz, scale, N, b0, b1, seed, R, s, i, P = task
    _, syn = O.sample(d, pxyz, seed, s, 1)
    Ri, _ = O.greedy(d, pxyz, scale, seed, s, i, 1, syn[0])
    LX, LZ = O.logicals(d)
    L = [0 * LX, LX, LX ^ LZ, LZ][P]
    ref = O.anneal_chain(d, pxyz, scale, O.LINEAR, N, b0, b1, seed, (s * R + i) * 4 + P, Ri ^ L)
    return Ri, O.class_bits(d, Ri), ref["best_E"]
