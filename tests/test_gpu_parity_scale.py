"""Oracle parity at scale, in the launch shape the benchmark times.

d = 11 workload: for each of the five noise points p in {0.10, ..., 0.22}
(eta = 100, 64 restarts, 1000 sweeps, linear beta 0.05 -> 20) one launch of
20,000 shots is decoded on the GPU exactly as a benchmark step decodes it
(greedy references, annealing of 256 chains per shot, decision), and a seeded
sample of 2000 of its shots per p is decoded by the oracle, shot by shot, on
every host core.  Classes, coset energies, all 256 chain minima, the class
bits of Q_i for all 64 references (the class of R_i R_1), recoveries and
failure flags must agree bit for bit
(Sec. "Simulation setting"; Alg. 7).  XZZX_PARITY_SHOTS_PER_P overrides the
sample size.

d = 31 workload (eta = 1000, 256 restarts, 1e4 sweeps, scale 4096): one
launch of 76 shots per noise point, for three noise points; 64 sampled
(shot, restart, coset) chains per point are re-annealed by the oracle from
its own greedy references, which must equal the GPU's references bit for bit.
"""
import os

import numpy as np
import pytest

import oracle as O
import oracle_pool
from layout import words_to_labels

pytestmark = pytest.mark.gpu

SHOTS_PER_P = int(os.environ.get("XZZX_PARITY_SHOTS_PER_P", "2000"))


@pytest.fixture(scope="module")
def X():
    from paper_2509_17837_gb300 import build
    build.build()
    import paper_2509_17837_gb300 as X
    return X


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def test_d11_parity_sampled_shots_every_p(X, torch):
    import bench
    d, R, S = bench.D, bench.RESTARTS, 20000
    code = X.Code(d)
    n_pick = min(SHOTS_PER_P, S)
    gpu, tasks, picks_by_p = [], [], []
    for pi, p in enumerate(bench.PS):
        seed = bench.SEED + pi
        noise = X.noise_from_eta(p, bench.ETA, 0, bench.SCALE)
        sched = X.Schedule(noise, bench.SWEEPS, bench.BETA0, bench.BETA1)
        shot0 = bench.rank_shot_base(0, 8, S) + 4 * S          # step 4 of rank 0
        err, syn = X.sample_errors(code, noise, seed, shot0, S)
        init, cbits = X.greedy_init(code, noise, seed, shot0, syn, R)
        a = X.anneal(code, sched, seed, shot0, init, want_cfg=False)
        out = X.decode_reduce(code, init, cbits, a["best_E"], true_errors=err)
        torch.cuda.synchronize()
        picks = np.sort(np.random.default_rng(1000 + pi).choice(S, n_pick, replace=False))
        idx = torch.as_tensor(picks, device=init.device)
        gpu.append(dict(cls=out["cls"][idx].cpu().numpy(), E4=out["E4"][idx].cpu().numpy(),
                        recovery=words_to_labels(out["recovery"][idx].cpu().numpy(), d * d),
                        fail=out["fail"][idx].cpu().numpy(),
                        chain_E=a["best_E"][idx].reshape(n_pick, -1).cpu().numpy(),
                        # class bits of Q_i, the class of R_i R_1 (Eq. coset_correspondence)
                        q_bits=(cbits[idx].cpu().numpy() & 3) ^ (cbits[idx][:, :1].cpu().numpy() & 3)))
        picks_by_p.append(picks)
        pxyz = (noise.px, noise.py, noise.pz)
        for lo, hi in oracle_pool.chunks(0, n_pick, 4 * oracle_pool.n_workers(n_pick)):
            tasks.append((pi, lo, hi, (d, pxyz, bench.SCALE, O.LINEAR, bench.SWEEPS, bench.BETA0, bench.BETA1,
                                       seed, R, 1, (shot0 + picks[lo:hi]).tolist())))
    results = oracle_pool.run(oracle_pool.decode_shots, [t[3] for t in tasks])
    mismatches = 0
    for (pi, lo, hi, _), ref in zip(tasks, results):
        g = {k: v[lo:hi] for k, v in gpu[pi].items()}
        for k in ("cls", "E4", "recovery", "fail", "chain_E", "q_bits"):
            bad = np.nonzero((g[k] != ref[k]).reshape(hi - lo, -1).any(1))[0]
            if len(bad):
                mismatches += len(bad)
                pytest.fail("p=%.2f: %s differs on shots %s" % (bench.PS[pi], k,
                                                                 (picks_by_p[pi][lo + bad[:5]]).tolist()))
    assert mismatches == 0
    print("d=11 parity: %d shots x %d p values, %d chains, 0 mismatches" % (n_pick, len(bench.PS),
                                                                          n_pick * len(bench.PS) * 4 * R))


def test_d31_parity_sampled_chains_three_p(X, torch):
    import bench
    d, R, N, b0, b1, scale, eta, seed = 31, 256, 10000, 0.02, 30.0, 4096, 1000.0, 0xD31
    S = 76
    code = X.Code(d)
    for p in (bench.LARGE_PS[0], bench.LARGE_PS[len(bench.LARGE_PS) // 2], bench.LARGE_PS[-1]):
        noise = X.noise_from_eta(p, eta, 0, scale)
        sched = X.Schedule(noise, N, b0, b1)
        err, syn = X.sample_errors(code, noise, seed, 0, S)
        init, cbits = X.greedy_init(code, noise, seed, 0, syn, R)
        a = X.anneal(code, sched, seed, 0, init, want_cfg=False)
        torch.cuda.synchronize()
        init_h, cb_h, best_E = init.cpu().numpy(), cbits.cpu().numpy(), a["best_E"].cpu().numpy()
        rng = np.random.default_rng(int(p * 1000))
        picks = [(int(s), int(i), int(P)) for s, i, P in zip(rng.integers(0, S, 64), rng.integers(0, R, 64),
                                                              rng.integers(0, 4, 64))]
        pxyz = (noise.px, noise.py, noise.pz)
        refs = oracle_pool.run(oracle_pool.anneal_one_chain, [(d, pxyz, scale, N, b0, b1, seed, R, s, i, P) for s, i, P in picks])
        for (s, i, P), (Ri, qb, bE) in zip(picks, refs):
            assert np.array_equal(words_to_labels(init_h[s, i], d * d), Ri), (p, s, i)
            assert cb_h[s, i] & 3 == qb, (p, s, i)
            assert best_E[s, i, P] == bE, (p, s, i, P)
