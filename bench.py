"""Benchmark of the XZZX simulated-annealing decoder on one GB300 (or N, weak scaling).

Workload (one step = one pass of the whole hot path over one batch):
  rotated d = 11 XZZX code (121 qubits, 120 generators), code-capacity noise
  with py = p eta/(eta+1), px = pz = p/(2(eta+1)), eta = 100, and one batch of
  --shots-per-p shots at each p in {0.10, 0.13, 0.16, 0.19, 0.22}; 64 greedy
  restarts per shot (256 chains), 1000 sweeps, linear beta 0.05 -> 20 (units
  of the Nishimori beta), energies at scale 1024.  Step k decodes shots
  [k*S, (k+1)*S) of every p, so --steps 5 with S = 20000 covers the full
  1e5 shots per p.  Inputs are sampled by the library on the device before the
  timed region; L2 is flushed between steps.

Printed JSON line: value = move attempts per second of the whole step (greedy
+ anneal + decision), plus shots/s, the anneal kernel's own rate and its
roofline, the oracle CPU baseline, end-to-end numbers through the C ABI with
host buffers, and SM clocks sampled during the timed region.

--impl reference times the oracle (plain single-threaded C++) on the host's
cores on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

D, ETA, PS, RESTARTS, SWEEPS, BETA0, BETA1, SCALE = 11, 100.0, (0.10, 0.13, 0.16, 0.19, 0.22), 64, 1000, 0.05, 20.0, 1024
SEED = 0xD11
I_ALG = 30  # integer instructions per move attempt in the algorithmic count
# Counters of the current anneal_kernel<11> from one ncu capture (None until
# the kernel has been captured since its last change): DRAM bytes (read +
# write) per chain, ALU-pipe lane instructions per move attempt
# (sm__inst_executed_pipe_alu x 32 / attempts; the ALU pipe takes 16 lanes per
# clock per SM sub-partition), all lane instructions per attempt
# (smsp__inst_executed x 32 / attempts) and shared-memory bank conflicts per
# shared wavefront.
ANNEAL_DRAM_BYTES_PER_CHAIN = 8.399872e6 / 1.024e6
ANNEAL_ALU_INST_PER_ATTEMPT = 12.12
ANNEAL_MEASURED = {"inst_per_attempt": 20.51, "alu_inst_per_attempt": ANNEAL_ALU_INST_PER_ATTEMPT,
                   "shared_bank_conflicts_per_wavefront": 1.2654e10 / 2.0863e10,
                   "source": "ncu capture of one anneal_kernel<11> launch of 4000 shots, "
                             "profiles/anneal_d11_ncu_full.md"}
# The same counters for the d=31 row kernel of the large workload, taken on
# its form before the group-by-group columns and the 128-register bound:
# DRAM traffic is therefore not reported for the current kernel.
ANNEAL_D31_DRAM_BYTES_PER_CHAIN = None
ANNEAL_D31_MEASURED = {"inst_per_attempt": 18.83, "alu_inst_per_attempt": 11.69,
                       "shared_bank_conflicts_per_wavefront": 5.7998e10 / 9.3272e10,
                       "dram_bytes_per_chain": 4.580864e6 / (57 * 1024),
                       "source": "ncu capture of one launch of the previous form of the d=31 row kernel "
                                 "(158 registers, 3 CTAs per SM), profiles/anneal_d31_ncu_full.md"}


def workload_config(shots_per_p, world):
    return {"workload": "d=11 rotated XZZX, eta=100, p in {0.10,0.13,0.16,0.19,0.22}, 64 restarts (256 chains)/shot, "
                        "1000 sweeps, linear beta 0.05->20, scale 1024",
            "code_distance": D, "restarts": RESTARTS, "sweeps": SWEEPS, "shots_per_p_per_step": shots_per_p,
            "p_values": list(PS), "eta": ETA, "global_batch": shots_per_p * len(PS) * world,
            "parallelism": "shots sharded across ranks" if world > 1 else "single GPU",
            "l2": "flushed between steps (512 MiB write)"}


def attempts_per_shot():
    return 4 * RESTARTS * SWEEPS * (D * D - 1)


def rank_shot_base(rank, n_steps, shots_per_step):
    """First shot index of a rank's own range.  Shots are independent and every
    draw is keyed by the absolute shot index, so ranks decode disjoint ranges
    with no data exchange (weak scaling)."""
    return rank * n_steps * shots_per_step


def max_over_ranks(values, dist, device):
    """Element-wise MAX of per-rank timings (the slowest rank sets the time)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def sum_over_ranks(values, dist, device):
    """Element-wise SUM over ranks (counts such as logical failures)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(x) for x in t]


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while the timed
    region runs (written to ``path``, a temporary file unless one is given)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, path, gpu_index):
        self.temporary = not path
        if self.temporary:
            import tempfile
            fd, path = tempfile.mkstemp(prefix="xzzx_clocks_", suffix=".csv")
            os.close(fd)
        self.path, self.gpu_index, self.proc = path, gpu_index, None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if self.temporary:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        top = max(sm)
        loaded = [x for x in sm if x >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def issue_peak(clocks, n_sm):
    """Integer issue peak in T lane-instructions/s (SMs x 4 SMSP x 32 lanes x
    the median SM clock sampled in the timed region), with its basis; (None,
    reason) when no clock was sampled, so the roofline is reported unmeasured
    rather than guessed."""
    f_mhz = (clocks or {}).get("sm_mhz")
    if not f_mhz:
        return None, "unmeasured: no SM clock samples (%s)" % ",".join((clocks or {}).get("reasons", []) or ["none"])
    return (n_sm * 4 * 32 * f_mhz * 1e6 / 1e12,
            "%d SMs x 4 SMSP x 32 lanes x %.0f MHz (median SM clock sampled in the timed region)" % (n_sm, f_mhz))


def roofline_record(rate_attempts, clocks, n_sm, **extra):
    peak, basis = issue_peak(clocks, n_sm)
    achieved = rate_attempts * I_ALG / 1e12
    rec = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s",
           "frac": (achieved / peak) if peak else None, "I_alg_per_attempt": I_ALG, "peak_basis": basis}
    rec.update(extra)
    return rec


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    import oracle as O
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    shots = args.ref_shots
    pxyz = O.noise_from_eta(0.16, ETA)
    err, syn = O.sample(D, pxyz, SEED, 0, shots * (args.steps + args.warmup))
    for w in range(args.warmup):
        O.decode(D, pxyz, SCALE, O.LINEAR, SWEEPS, BETA0, BETA1, SEED, w * shots, RESTARTS,
                 syn[w * shots:(w + 1) * shots])
    t0 = time.perf_counter()
    for k in range(args.steps):
        s0 = (args.warmup + k) * shots
        O.decode(D, pxyz, SCALE, O.LINEAR, SWEEPS, BETA0, BETA1, SEED, s0, RESTARTS, syn[s0:s0 + shots])
    dt = time.perf_counter() - t0
    att = attempts_per_shot() * shots * args.steps / dt
    sample = "%d shots of d=11 p=0.16 per step, single-threaded oracle" % shots
    print(json.dumps({
        "impl": "reference", "metric": "move-attempts/s and decoded shots/s at d=11 (64 restarts); serve p50/p99 latency",
        "value": att, "unit": "move-attempts/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic (library sampler, seeded)",
        "config": dict(workload_config(shots, 1), global_batch=shots, parallelism="one host core (the oracle)",
                       shots_per_p_per_step=None, sample=sample, l2="n/a (host)"),
        "shots_per_s": shots * args.steps / dt,
        "cpu_baseline": {"value": att, "unit": "move-attempts/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": att, "unit": "move-attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# --------------------------------------------------------------------------- CPU baseline (oracle)
def _oracle_worker(args):
    shot0, shots = args
    import oracle as O
    pxyz = O.noise_from_eta(0.16, ETA)
    err, syn = O.sample(D, pxyz, SEED, shot0, shots)
    O.decode(D, pxyz, SCALE, O.LINEAR, SWEEPS, BETA0, BETA1, SEED, shot0, RESTARTS, syn, err)
    return shots


def cpu_baseline_all_cores(shots_per_core):
    """The oracle as independent single-threaded processes on every host core,
    over disjoint shot ranges (spawned, so no CUDA state is inherited)."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    import oracle.build
    oracle.build.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(n) as pool:
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_worker, [(1000 + k * shots_per_core, shots_per_core) for k in range(n)]))
        dt = time.perf_counter() - t0
    return {"value": attempts_per_shot() * done / dt, "unit": "move-attempts/s", "cores": n, "kind": "oracle",
            "sample": "%d processes x %d shots of d=11 p=0.16, %.1f s wall" % (n, shots_per_core, dt),
            "shots_per_s": done / dt}


def _parity_worker(task):
    """Oracle decode of listed d=11 shots of one noise point, shot by shot."""
    pi, shots = task
    import numpy as np
    import oracle as O
    pxyz = O.noise_from_eta(PS[pi], ETA)
    out = {k: [] for k in ("cls", "E4", "recovery", "fail")}
    for s in shots:
        err, syn = O.sample(D, pxyz, SEED + pi, int(s), 1)
        r = O.decode(D, pxyz, SCALE, O.LINEAR, SWEEPS, BETA0, BETA1, SEED + pi, int(s), RESTARTS, syn, err)
        for k in out:
            out[k].append(r[k][0])
    return pi, list(shots), {k: np.array(v) for k, v in out.items()}


class ParityLeg:
    """Oracle parity on a seeded sample of the shots of the last timed step.

    The oracle decodes the sampled shots in spawned single-threaded processes
    on all host cores but one while the GPU runs; afterwards each shot's
    class, coset energies, recovery and failure flag are compared with the
    GPU's outputs element by element."""

    def __init__(self, shot_first, S, per_p, seed=0x9A7):
        import numpy as np
        self.picks = [np.sort(np.random.default_rng(seed + pi).choice(S, min(per_p, S), replace=False))
                      for pi in range(len(PS))]
        self.shot_first, self.per_p = shot_first, per_p
        self.pool = self.result = None
        if per_p <= 0:
            return
        import multiprocessing as mp
        import oracle.build
        oracle.build.build()
        n = max(1, (os.cpu_count() or 2) - 1)
        tasks = []
        for pi, pk in enumerate(self.picks):
            shots = (shot_first[pi] + pk).tolist()
            step = max(1, (len(PS) * per_p) // (3 * n))
            tasks += [(pi, shots[j:j + step]) for j in range(0, len(shots), step)]
        self.cores = n
        self.t0 = time.perf_counter()
        self.pool = mp.get_context("spawn").Pool(n)
        self.result = self.pool.map_async(_parity_worker, tasks, chunksize=1)

    def compare(self, gpu_outs, words):
        """gpu_outs[pi]: dict of the last step's device outputs for noise point pi."""
        if self.pool is None:
            return None
        import numpy as np
        parts = self.result.get()
        wall = time.perf_counter() - self.t0
        self.pool.close()
        self.pool.join()
        host = [{k: v.cpu().numpy() for k, v in o.items() if v is not None} for o in gpu_outs]
        mism, shots, bad = 0, 0, []
        for pi, shot_ids, ref in parts:
            g = host[pi]
            rows = [int(s) - self.shot_first[pi] for s in shot_ids]
            rec = g["recovery"][rows].view(np.uint32)
            x = np.unpackbits(rec[:, :words].view(np.uint8), axis=1, bitorder="little")[:, :D * D]
            z = np.unpackbits(rec[:, words:].view(np.uint8), axis=1, bitorder="little")[:, :D * D]
            lab = (x << 1) | z
            ok = ((g["cls"][rows] == ref["cls"]) & (g["E4"][rows] == ref["E4"]).all(1) &
                  (lab == ref["recovery"]).all(1) & (g["fail"][rows] == ref["fail"]))
            shots += len(rows)
            mism += int((~ok).sum())
            bad += [int(s) for s, o in zip(shot_ids, ok) if not o][:4]
        return {"shots": shots, "mismatches": mism, "compared": "cls, E4 (4 coset minima), recovery, fail",
                "source": "seeded sample of the last timed step's shots, %d per p" % self.per_p,
                "oracle_processes": self.cores, "oracle_wall_s": wall, "first_mismatched_shots": bad}


def cpu_baseline(shots):
    import oracle as O
    pxyz = O.noise_from_eta(0.16, ETA)
    err, syn = O.sample(D, pxyz, SEED, 0, shots)
    t0 = time.perf_counter()
    O.decode(D, pxyz, SCALE, O.LINEAR, SWEEPS, BETA0, BETA1, SEED, 0, RESTARTS, syn, err)
    dt = time.perf_counter() - t0
    return {"value": attempts_per_shot() * shots / dt, "unit": "move-attempts/s", "cores": 1, "kind": "oracle",
            "sample": "%d shots of d=11 p=0.16 (full 64 restarts x 1000 sweeps), single thread, %.1f s" % (shots, dt),
            "shots_per_s": shots / dt}


# --------------------------------------------------------------------------- uneven batch (NEXT f1)
UNEVEN_DS = (5, 7, 9, 13, 17, 21)
UNEVEN_R = {5: 16, 7: 16, 9: 32, 13: 32, 17: 64, 21: 64}
UNEVEN_N = {5: 500, 7: 500, 9: 1000, 13: 1000, 17: 2000, 21: 2000}
UNEVEN_ETAS = (1.0, 10.0, 100.0)
UNEVEN_PS = tuple(round(0.08 + 0.005 * k, 3) for k in range(25))   # [0.08, 0.20] on a 0.005 grid


def uneven_segments(X, total_shots, seed, scale_shots=1.0, scale_sweeps=1.0):
    """Shots of distances {5,7,9,13,17,21} in equal numbers; eta and p drawn per
    shot from the seed (p on a 0.005 grid: 75 noise classes per distance);
    shots bucketed into homogeneous segments with disjoint shot indices.
    scale_shots / scale_sweeps shrink the batch for the autotuner: fewer
    sweeps keep every distance's chunk count, so the waves and tails the forms
    differ on keep their shape while each run is shorter."""
    import numpy as np
    rng = np.random.default_rng(seed)
    per_d = total_shots // len(UNEVEN_DS)
    segs, shot_base = [], 0
    codes, scheds = {}, {}
    for d in UNEVEN_DS:
        eta_i = rng.integers(0, len(UNEVEN_ETAS), per_d)
        p_i = rng.integers(0, len(UNEVEN_PS), per_d)
        counts = np.bincount(eta_i * len(UNEVEN_PS) + p_i, minlength=len(UNEVEN_ETAS) * len(UNEVEN_PS))
        codes[d] = X.Code(d)
        for cls, n in enumerate(counts):
            n = int(round(n * scale_shots))
            if n == 0:
                continue
            eta, p = UNEVEN_ETAS[cls // len(UNEVEN_PS)], UNEVEN_PS[cls % len(UNEVEN_PS)]
            noise = X.noise_from_eta(p, eta)
            key = (d, eta, p)
            if key not in scheds:
                scheds[key] = X.Schedule(noise, max(1, int(round(UNEVEN_N[d] * scale_sweeps))), BETA0, BETA1)
            err, syn = X.sample_errors(codes[d], noise, seed, shot_base, n)
            segs.append(dict(code=codes[d], noise=noise, sched=scheds[key], shot0=shot_base, syndromes=syn,
                             true_errors=err, restarts=UNEVEN_R[d]))
            shot_base += n
    return segs


def run_uneven(args):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_17837_gb300 as X
    from paper_2509_17837_gb300 import autotune
    seed = 0xF1
    segs = uneven_segments(X, args.uneven_shots, seed)
    # the tuner times a batch of the same shots (at most 60k) with a tenth of
    # the sweeps: the same chunks per distance, so the same waves and tails
    tune_scale = min(1.0, 60000.0 / args.uneven_shots)
    tune_segs = uneven_segments(X, args.uneven_shots, seed, scale_shots=tune_scale, scale_sweeps=0.1)
    class GraphForm:
        """A tuning candidate run the way the benchmark times it: modes 0, 3
        and 4 as captured graphs (one batch per mode, created on first use)."""

        def __init__(self, c, o, nt, u):
            self.knobs, self.batches = (c, o, nt, u), {}

        def run(self, mode, stream):
            c, o, nt, u = self.knobs
            if mode not in self.batches:
                self.batches[mode] = X.Batch(tune_segs, seed, ctas_per_sm=c, order=o, chains_per_cta=nt,
                                             sweep_unroll=u, graph_mode=mode if mode in (3, 4) else 0)
            b = self.batches[mode]
            with torch.cuda.stream(stream):
                b.run_graph(stream) if mode in (0, 3, 4) else b.run(mode, stream)

        def close(self):
            for b in self.batches.values():
                b.close()

    tune_stream = torch.cuda.Stream()
    cfg, timings = autotune.tune(GraphForm, tune_segs, reps=3, use_cache=False, stream=tune_stream,
                                 sync=tune_stream.synchronize)
    knobs = lambda key: tuple(int(x) for x in key.split(","))
    best_of = lambda modes: knobs(min((k for k in timings if knobs(k)[0] in modes), key=timings.get))
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        stream.synchronize()
        ms = 0.0
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
            stream.synchronize()
            ms += e0.elapsed_time(e1)
        return ms / steps

    def form(mode, cps, order, nt, u):
        """A batch in one of the forms, and the call that runs it (modes 0 and 3
        as captured graphs)."""
        b = X.Batch(segs, seed, ctas_per_sm=cps, order=order, graph_mode=mode if mode in (3, 4) else 0,
                    chains_per_cta=nt, sweep_unroll=u)
        run = (lambda: b.run_graph(stream)) if mode in (0, 3, 4) else (lambda: b.run(mode, stream))
        return b, run

    sampler = ClockSampler(args.clocks_csv, dev)
    sampler.start()
    forms = {"tuned": cfg, "persistent": best_of((0,)), "concurrent": best_of((3,)),
             "class_persistent": best_of((4,)), "plain": (1, 0, 0, 128, 1)}
    ms, outs, info = {}, {}, None
    for name, (mode, cps, order, nt, u) in forms.items():
        b, run = form(mode, cps, order, nt, u)
        with torch.cuda.stream(stream):
            ms[name] = timed(run, args.steps, args.warmup)
        stream.synchronize()
        outs[name] = [{k: (v.clone() if v is not None else None) for k, v in o.items()} for o in b.outputs]
        if name == "tuned":
            info = b.info()
        b.close()
    clocks = sampler.stop()
    ref = outs["plain"]
    same = all(torch.equal(a[k], r[k]) for name in outs for a, r in zip(outs[name], ref) for k in r
               if r[k] is not None)
    fails = sum(int(o["fail"].sum()) for o in ref)
    shots = info["total_shots"]
    props = torch.cuda.get_device_properties(dev)
    att = info["move_attempts"] / (ms["tuned"] / 1e3)
    form_rec = lambda name: {"cfg": dict(zip(("mode", "ctas_per_sm", "order", "chains_per_cta", "sweep_unroll"),
                                             forms[name])),
                             "ms_per_step": ms[name], "shots_per_s": shots / (ms[name] / 1e3),
                             "speedup_vs_plain": ms["plain"] / ms[name]}
    print(json.dumps({
        "metric": "decoded shots/s, uneven batch (d in {5,7,9,13,17,21}; tuned batched form vs one launch per distance)",
        "value": shots / (ms["tuned"] / 1e3), "unit": "shots/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms["tuned"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded per-shot eta and p; library sampler)",
        "config": {"workload": "uneven batch: %d shots, distances {5,7,9,13,17,21} equal, eta in {1,10,100}, "
                               "p in [0.08,0.20] (0.005 grid), restarts {16,16,32,32,64,64}, sweeps "
                               "{500,500,1000,1000,2000,2000}, linear beta 0.05->20" % shots,
                   "segments": info["n_segments"], "chunks": info["n_chunks"],
                   "tuned_cfg": form_rec("tuned")["cfg"],
                   "modes": "0 persistent (one chain per thread, chunk queue), 1 one launch per distance, 2 per "
                            "distance with one warp per chain, 3 per-distance launches on forked streams, 4 one "
                            "persistent launch per distance class on forked streams; 0, 3 and 4 replayed as "
                            "captured CUDA graphs",
                   "autotune": {"batch_shots": int(sum(int(sg["syndromes"].shape[0]) for sg in tune_segs)),
                                "sweeps": "a tenth of the workload's",
                                "timings_s": timings},
                   "l2": "flushed between steps"},
        "move_attempts_per_s": att, "forms": {name: form_rec(name) for name in forms},
        "speedup_vs_plain": ms["plain"] / ms["tuned"], "identical_outputs": bool(same),
        "logical_failures": fails, "clocks": clocks,
        "roofline": roofline_record(att, clocks, props.multi_processor_count, traffic=None,
                                    kernel="annealing launches of the tuned form (all distances)")}))


# --------------------------------------------------------------------------- serving (NEXT f2)
SERVE_DS = (5, 9, 13, 17, 21, 25)
SERVE_RATES = (1e3, 3e3, 1e4, 3e4, 1e5, 3e5, 1e6)


def run_serve(args):
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_17837_gb300 as X
    seed, R, N = 0x5E5E, 32, 1000
    sv = X.Server(seed, R, N, BETA0, BETA1, max_batch=args.serve_max_batch, n_slots=args.serve_slots,
                  queue_capacity=1 << 22, hbm_budget_bytes=1 << 30, resident_waves=args.serve_waves)
    noise = X.noise_from_eta(0.15, ETA)
    cids = [sv.add_class(d, noise) for d in SERVE_DS]
    sv.start()
    # a pool of syndromes per distance, sampled on the device by the library
    pool = {}
    for d in SERVE_DS:
        code = X.Code(d)
        _, syn = X.sample_errors(code, noise, seed, 0, 4096, want_errors=False)
        a = np.zeros((4096, 32), np.uint32)
        a[:, :code.syn_words] = syn.cpu().numpy().view(np.uint32)
        pool[d] = a
    rng = np.random.default_rng(seed)
    points, next_id = [], 1 << 40

    def run_point(rate, n):
        nonlocal next_id
        which = rng.integers(0, len(SERVE_DS), n)
        syn = np.stack([pool[SERVE_DS[w]][rng.integers(0, 4096)] for w in which])
        ids = np.arange(next_id, next_id + n, dtype=np.uint64)
        next_id += n
        arrivals = np.cumsum(rng.exponential(1e6 / rate, n))
        sv.stats(reset=True)
        t0 = time.perf_counter()
        sv.replay(ids, [cids[w] for w in which], syn, arrivals)
        got = 0
        while got < n and time.perf_counter() - t0 < 600:
            got += len(sv.poll(cap=1 << 16, timeout_ms=100))
        makespan = time.perf_counter() - t0
        st = sv.stats()
        return {"offered_req_per_s": rate, "requests": n, "completed": st["completed"],
                "throughput_req_per_s": st["completed"] / makespan, "p50_ms": st["p50_us"] / 1e3,
                "p99_ms": st["p99_us"] / 1e3, "max_ms": st["max_us"] / 1e3, "mean_batch": st["mean_batch"],
                "batches": st["batches"], "rejected": st["rejected"]}

    run_point(1e4, 200)  # warm-up
    for rate in SERVE_RATES:
        n = int(min(max(rate * args.serve_seconds, 400), args.serve_max_requests))
        points.append(run_point(rate, n))
    sv.close()
    sat = max(points, key=lambda x: x["throughput_req_per_s"])
    mean_att = np.mean([4 * R * N * (d * d - 1) for d in SERVE_DS])
    print(json.dumps({
        "metric": "serve p50/p99 latency vs offered load (continuous batching, mixed distances)",
        "value": sat["throughput_req_per_s"], "unit": "req/s at saturation", "n_gpus": 1,
        "steps": len(points), "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (library sampler, seeded; Poisson arrivals)",
        "config": {"workload": "serving: Poisson single-shot requests, d uniform over {5,9,13,17,21,25}, eta=100, "
                               "p=0.15, 32 restarts, 1000 sweeps, linear beta 0.05->20",
                   "max_batch": args.serve_max_batch, "slots": args.serve_slots, "hbm_budget_bytes": 1 << 30,
                   "resident_waves": args.serve_waves or 2},
        "points": points, "saturation_move_attempts_per_s": sat["throughput_req_per_s"] * mean_att}))


# --------------------------------------------------------------------------- large distance (NEXT f4)
LARGE_PS = (0.15, 0.18, 0.21, 0.24, 0.27, 0.30)


def run_large(args):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_17837_gb300 as X
    from paper_2509_17837_gb300 import stats
    d, R, N, b0, b1, scale, eta, seed = 31, 256, 10000, 0.02, 30.0, 4096, 1000.0, 0xD31
    S = args.large_shots_per_p
    code = X.Code(d)
    stream = torch.cuda.current_stream()
    cases = []
    for i, p in enumerate(LARGE_PS):
        noise = X.noise_from_eta(p, eta, 0, scale)
        sched = X.Schedule(noise, N, b0, b1)
        err, syn = X.sample_errors(code, noise, seed + i, 0, S * (args.steps + 1))
        cases.append((noise, sched, seed + i, err, syn))
    ws = torch.empty(X.decode_workspace_size(code, S, R), dtype=torch.uint8, device="cuda")
    fails = [0] * len(cases)

    def step(k):
        ms = 0.0
        for ci, (noise, sched, sd, err, syn) in enumerate(cases):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = X.decode_batch(code, noise, sched, sd, k * S, syn[k * S:(k + 1) * S], R,
                                 true_errors=err[k * S:(k + 1) * S], workspace=ws, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            fails[ci] += int(out["fail"].sum())
        return ms

    step(0)
    fails = [0] * len(cases)
    sampler = ClockSampler(args.clocks_csv, torch.cuda.current_device())
    sampler.start()
    ms = sum(step(k + 1) for k in range(args.steps)) / args.steps
    clocks = sampler.stop()
    shots = S * len(LARGE_PS)
    att = shots * 4 * R * N * (d * d - 1) / (ms / 1e3)
    props = torch.cuda.get_device_properties(0)

    # The same annealing launch (first p, step 1) with one warp per chain and
    # colour-parallel lanes, against one thread per chain: identical chain
    # minima, and each mapping's rate.
    noise, sched, sd, err, syn = cases[0]
    init, _ = X.greedy_init(code, noise, sd, S, syn[S:2 * S], R)
    mapping = {}
    best = {}
    for name, per_warp in (("thread_per_chain", False), ("warp_per_chain", True)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        a = X.anneal(code, sched, sd, S, init, want_cfg=False, per_warp=per_warp, stream=stream)
        e1.record(stream)
        e1.synchronize()
        best[name] = a["best_E"]
        mapping[name] = {"anneal_ms": e0.elapsed_time(e1),
                         "attempts_per_s": S * 4 * R * N * (d * d - 1) / (e0.elapsed_time(e1) / 1e3)}
    mapping["identical_chain_minima"] = bool(torch.equal(best["thread_per_chain"], best["warp_per_chain"]))

    # Occupancy sweep: the same shots with a given number of chains in flight
    # per SM (CTAs per SM x chains per CTA), one chain per thread as one
    # persistent launch, then one chain per warp.  Decisions must equal the
    # plain decode of the same shots.
    ref = X.decode_batch(code, noise, sched, sd, S, syn[S:2 * S], R, true_errors=err[S:2 * S], stream=stream)
    occupancy = []
    if not args.no_occupancy_sweep:
        for nt, cps in ((128, 1), (128, 2), (128, 3), (256, 1)):
            seg = dict(code=code, noise=noise, sched=sched, shot0=S, syndromes=syn[S:2 * S], restarts=R,
                       true_errors=err[S:2 * S])
            b = X.Batch([seg], sd, ctas_per_sm=cps, chains_per_cta=nt)
            b.run(0, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(0, stream)
            e1.record(stream)
            e1.synchronize()
            o = b.outputs[0]
            same = all(torch.equal(o[k], ref[k]) for k in ("cls", "E4", "recovery", "fail"))
            info = b.info()
            in_flight = info["persistent_grid"] * nt // props.multi_processor_count
            occupancy.append({"mapping": "thread_per_chain", "chains_per_cta": nt, "ctas_per_sm": cps,
                              "chains_in_flight_per_sm": in_flight,
                              "ms": e0.elapsed_time(e1),
                              "attempts_per_s": info["move_attempts"] / (e0.elapsed_time(e1) / 1e3),
                              "identical_decisions": bool(same)})
            b.close()
        # One warp per chain (mode 2, 4 chains per CTA): resident CTAs per SM
        # capped by padding each CTA's shared memory (0 = the register limit).
        for cps in (2, 4, 8, 0):
            seg = dict(code=code, noise=noise, sched=sched, shot0=S, syndromes=syn[S:2 * S], restarts=R,
                       true_errors=err[S:2 * S])
            b = X.Batch([seg], sd, ctas_per_sm=cps)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(2, stream)
            e1.record(stream)
            e1.synchronize()
            o = b.outputs[0]
            same = all(torch.equal(o[k], ref[k]) for k in ("cls", "E4", "recovery", "fail"))
            info = b.info()
            occupancy.append({"mapping": "warp_per_chain", "chains_per_cta": 4, "ctas_per_sm_cap": cps,
                              "chains_in_flight_per_sm": 4 * info["warp_ctas_per_sm"],
                              "ms": e0.elapsed_time(e1),
                              "attempts_per_s": info["move_attempts"] / (e0.elapsed_time(e1) / 1e3),
                              "identical_decisions": bool(same)})
            b.close()
    print(json.dumps({
        "metric": "move-attempts/s and decoded shots/s at d=31 (256 restarts, 1e4 sweeps)",
        "value": att, "unit": "move-attempts/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (library sampler, seeded)",
        "config": {"workload": "d=31 rotated XZZX, eta=1000, p in {0.15..0.30}, 256 restarts (1024 chains)/shot, "
                               "1e4 sweeps, linear beta 0.02->30, scale 4096", "shots_per_p_per_step": S},
        "shots_per_s": shots / (ms / 1e3), "shots_timed": shots * args.steps,
        "logical_error_rates": [stats.ler_record(p, f, S * args.steps) for p, f in zip(LARGE_PS, fails)],
        "chain_mapping": mapping, "occupancy_sweep": occupancy, "clocks": clocks,
        "roofline": roofline_record(att, clocks, props.multi_processor_count,
                                    traffic=(None if ANNEAL_D31_DRAM_BYTES_PER_CHAIN is None
                                             else ANNEAL_D31_DRAM_BYTES_PER_CHAIN * S * R * 4),
                                    kernel="anneal_kernel_rows4<31>", measured_per_attempt=ANNEAL_D31_MEASURED)}))


# --------------------------------------------------------------------------- logical error rate curves
LER_D = (5, 7, 9)
LER_GRID = {1.0: (0.12, 0.14, 0.16, 0.18, 0.20, 0.22, 0.24), 5.0: (0.14, 0.16, 0.18, 0.20, 0.22, 0.24, 0.26),
            10.0: (0.06, 0.08, 0.10, 0.12, 0.14, 0.16, 0.18)}
# finite-size threshold estimates the paper states for its own SA decoder (context only)
LER_PAPER_PTH = {1.0: 0.18, 5.0: 0.2, 10.0: 0.11}


def crossing(ps, lo_d, hi_d):
    """p where LER(hi_d) - LER(lo_d) changes sign (linear interpolation), or None."""
    diff = [h - l for l, h in zip(lo_d, hi_d)]
    for k in range(len(ps) - 1):
        if diff[k] < 0 <= diff[k + 1]:
            return ps[k] + (ps[k + 1] - ps[k]) * (-diff[k]) / (diff[k + 1] - diff[k])
    return None


def run_ler(args):
    """Logical error rate vs p for d = 5, 7, 9 under depolarizing, 1:5:1 and
    1:10:1 Y-biased noise with the paper's decoder settings (N_beta = 100 log
    schedule 0.9 -> 1.0 beta_N, N_SA = 100, randomised greedy references), for
    the colour sweep and the literal random-site / per-attempt-minimum form."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_17837_gb300 as X
    from paper_2509_17837_gb300 import stats
    NSA, NB, shots, chunk = 100, 100, args.ler_shots, 25000
    layout = X.LAYOUT_PLANAR if args.layout == "planar" else X.LAYOUT_ROTATED
    forms = {"colour": (X.ORDER_COLOUR, X.EMIN_PER_PHASE), "literal": (X.ORDER_RANDOM_SITE, X.EMIN_PER_ATTEMPT)}
    curves, anneal_ms, attempts, total_shots = {}, {k: 0.0 for k in forms}, {k: 0 for k in forms}, 0
    t_wall = time.perf_counter()
    for eta, ps in LER_GRID.items():
        for d in LER_D:
            code = X.Code(d, layout)
            for pi, p in enumerate(ps):
                noise = X.noise_from_eta(p, eta, X.CONVENTION_PAPER, 1024)
                sched = X.Schedule(noise, NB, 0.9, 1.0, X.PAPER_LOG)
                seed = 0x1E2 + 1000 * int(eta) + pi
                for form, (order, emin) in forms.items():
                    fails = 0
                    for s0 in range(0, shots, chunk):
                        n = min(chunk, shots - s0)
                        err, syn = X.sample_errors(code, noise, seed, s0, n)
                        init, cb = X.greedy_init(code, noise, seed, s0, syn, NSA)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        a = X.anneal(code, sched, seed, s0, init, want_cfg=False, order=order, emin=emin)
                        e1.record()
                        r = X.decode_reduce(code, init, cb, a["best_E"], true_errors=err)
                        fails += int(r["fail"].sum())
                        anneal_ms[form] += e0.elapsed_time(e1)
                    attempts[form] += shots * NSA * 4 * NB * code.n_stab
                    total_shots += shots
                    curves.setdefault(form, {}).setdefault("%g" % eta, {}).setdefault(str(d), []).append(
                        stats.ler_record(p, fails, shots))
    wall = time.perf_counter() - t_wall
    cross = {form: {e: {"d5_d7": crossing(LER_GRID[float(e)], [r["ler"] for r in c["5"]], [r["ler"] for r in c["7"]]),
                        "d7_d9": crossing(LER_GRID[float(e)], [r["ler"] for r in c["7"]], [r["ler"] for r in c["9"]])}
                    for e, c in fc.items()} for form, fc in curves.items()}
    print(json.dumps({
        "metric": "logical error rate vs p (d=5,7,9) with the paper's decoder settings",
        "value": total_shots / wall, "unit": "decoded shots/s (whole sweep, wall clock)", "n_gpus": 1,
        "steps": 1, "warmup": 0, "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (library sampler, seeded)",
        "config": {"workload": "%s lattice, d in {5,7,9}, eta in {1,5,10} (px:py:pz = 1:eta:1), 7 values of p each, "
                               "%d shots per point, N_SA=100, N_beta=100, log schedule 0.9->1.0 beta_N"
                               % (args.layout, shots),
                   "forms": {"colour": "colour sweep, minimum per colour phase",
                             "literal": "random generator per attempt, minimum per attempt (Alg. 2 / Alg. 3)"}},
        "anneal_attempts_per_s": {k: attempts[k] / (anneal_ms[k] / 1e3) for k in forms},
        "curves": curves, "crossings": cross, "paper_threshold_estimates": LER_PAPER_PTH}))


# --------------------------------------------------------------------------- our arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--shots-per-p", type=int, default=20000)
    ap.add_argument("--ref-shots", type=int, default=2)
    ap.add_argument("--cpu-shots", type=int, default=18)
    ap.add_argument("--cpu-shots-per-core", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-greedy-only", action="store_true")
    ap.add_argument("--parity-shots-per-p", type=int, default=100)
    ap.add_argument("--clocks-csv", default=None, help="where to keep the nvidia-smi clock samples")
    ap.add_argument("--workload", default="d11", choices=["d11", "uneven", "serve", "large", "ler"])
    ap.add_argument("--ler-shots", type=int, default=100000)
    ap.add_argument("--layout", default="rotated", choices=["rotated", "planar"])
    ap.add_argument("--large-shots-per-p", type=int, default=76)  # one wave: 152 SMs x 4 CTAs x 128 chains
    ap.add_argument("--no-occupancy-sweep", action="store_true")
    ap.add_argument("--uneven-shots", type=int, default=1000000)
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-max-requests", type=int, default=30000)
    ap.add_argument("--serve-max-batch", type=int, default=1024)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-waves", type=int, default=0)
    args = ap.parse_args()
    if args.workload == "uneven" and args.impl == "ours":
        return run_uneven(args)
    if args.workload == "serve" and args.impl == "ours":
        return run_serve(args)
    if args.workload == "large" and args.impl == "ours":
        return run_large(args)
    if args.workload == "ler" and args.impl == "ours":
        return run_ler(args)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_17837_gb300 as X
    from paper_2509_17837_gb300 import stats

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    S = args.shots_per_p
    n_steps = args.warmup + args.steps
    code = X.Code(D)
    stream = torch.cuda.current_stream()
    cases = []
    for pi, p in enumerate(PS):
        noise = X.noise_from_eta(p, ETA, 0, SCALE)
        sched = X.Schedule(noise, SWEEPS, BETA0, BETA1)
        seed = SEED + pi
        # rank r decodes its own shot range: shots are independent (weak scaling)
        shot_base = rank_shot_base(rank, n_steps, S)
        err, syn = X.sample_errors(code, noise, seed, shot_base, n_steps * S)
        cases.append(dict(p=p, noise=noise, sched=sched, seed=seed, shot_base=shot_base, err=err, syn=syn))
    w2 = 2 * code.words
    init = torch.empty((S, RESTARTS, w2), dtype=torch.int32, device=dev)
    cbits = torch.empty((S, RESTARTS), dtype=torch.uint8, device=dev)
    chain_E = torch.empty((S, RESTARTS, 4), dtype=torch.int32, device=dev)
    outs = [dict(cls=torch.empty(S, dtype=torch.uint8, device=dev), E4=torch.empty((S, 4), dtype=torch.int32, device=dev),
                 recovery=torch.empty((S, w2), dtype=torch.int32, device=dev),
                 fail=torch.empty(S, dtype=torch.uint8, device=dev)) for _ in PS]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(k, record):
        times = []
        for c, o in zip(cases, outs):
            s0 = k * S
            syn = c["syn"][s0:s0 + S]
            err = c["err"][s0:s0 + S]
            e = [ev() for _ in range(4)]
            e[0].record(stream)
            X.greedy_init(code, c["noise"], c["seed"], c["shot_base"] + s0, syn, RESTARTS, init=init, cbits=cbits,
                          stream=stream)
            e[1].record(stream)
            X.anneal(code, c["sched"], c["seed"], c["shot_base"] + s0, init, want_cfg=False, best_E=chain_E,
                     stream=stream)
            e[2].record(stream)
            res = X.decode_reduce(code, init, cbits, chain_E, true_errors=err, stream=stream)
            e[3].record(stream)
            o["fail"] = res["fail"]
            o["res"] = res
            times.append(e)
        return times

    # oracle parity on a sample of the last timed step's shots, computed on the
    # host cores while the GPU runs (rank 0)
    parity = ParityLeg([c["shot_base"] + (n_steps - 1) * S for c in cases], S,
                       args.parity_shots_per_p if rank == 0 else 0)
    for k in range(args.warmup):
        step(k, False)
    barrier()
    sampler = ClockSampler(args.clocks_csv, dev)
    if rank == 0:
        sampler.start()
        time.sleep(0.5)
    barrier()
    t_wall = time.perf_counter()
    all_ev = []
    fails = [0] * len(PS)
    fail_hist = []
    for k in range(args.warmup, n_steps):
        flush.fill_(k & 0xFF)  # evict L2 between steps (outside the per-step events)
        all_ev.append(step(k, True))
        fail_hist.append([o["fail"] for o in outs])  # each step's reduce returns fresh tensors
    barrier()
    fail_dev = [sum(int(h[i].sum()) for h in fail_hist) for i in range(len(PS))]
    if world > 1:
        fail_dev = [int(f) for f in sum_over_ranks([float(f) for f in fail_dev], dist, dev)]
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop() if rank == 0 else None
    g_ms = a_ms = r_ms = 0.0
    for st in all_ev:
        for e in st:
            g_ms += e[0].elapsed_time(e[1])
            a_ms += e[1].elapsed_time(e[2])
            r_ms += e[2].elapsed_time(e[3])
    step_ms = (g_ms + a_ms + r_ms) / args.steps
    if world > 1:
        step_ms, a_ms_max = max_over_ranks([step_ms, a_ms], dist, dev)
    else:
        a_ms_max = a_ms
    shots_per_step = S * len(PS) * world
    att_per_step = shots_per_step * attempts_per_shot()
    value = att_per_step / (step_ms / 1e3)
    anneal_launches = args.steps * len(PS)
    anneal_ms_per_launch = a_ms_max / anneal_launches
    anneal_rate = S * attempts_per_shot() / (anneal_ms_per_launch / 1e3)  # per GPU

    result = None
    last_outs = [o["res"] for o in outs]
    if rank == 0:
        props = torch.cuda.get_device_properties(dev)
        n_sm = props.multi_processor_count
        f_mhz = (clocks or {}).get("sm_mhz")
        roof = roofline_record(
            anneal_rate, clocks, n_sm,
            traffic=None if ANNEAL_DRAM_BYTES_PER_CHAIN is None else ANNEAL_DRAM_BYTES_PER_CHAIN * S * RESTARTS * 4,
            kernel="anneal_kernel<11>",
            measured_per_attempt=ANNEAL_MEASURED,
            secondary_alu_pipe=None if not (f_mhz and ANNEAL_ALU_INST_PER_ATTEMPT) else {
                "alu_inst_per_attempt": ANNEAL_ALU_INST_PER_ATTEMPT,
                "peak_attempts_per_s": n_sm * 4 * 16 * f_mhz * 1e6 / ANNEAL_ALU_INST_PER_ATTEMPT,
                "frac": anneal_rate / (n_sm * 4 * 16 * f_mhz * 1e6 / ANNEAL_ALU_INST_PER_ATTEMPT)})
        result = {
            "metric": "move-attempts/s and decoded shots/s at d=11 (64 restarts); serve p50/p99 latency",
            "value": value, "unit": "move-attempts/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic (code-capacity noise sampled on device by the library, seeded)",
            "config": workload_config(S, world),
            "shots_per_s": shots_per_step / (step_ms / 1e3),
            "anneal_attempts_per_s_per_gpu": anneal_rate,
            "kernel_ms_per_step": {"greedy": g_ms / args.steps, "anneal": a_ms / args.steps,
                                   "reduce": r_ms / args.steps},
            "roofline": roof,
            "clocks": clocks, "gpu_launches": 3 * len(PS) * args.steps,
            "logical_error_rates": [stats.ler_record(p, f, S * args.steps * world) for p, f in zip(PS, fail_dev)],
            "wall_s_timed_region": wall,
        }
    # ---------------------------------------------------------------- greedy-only decisions (0 sweeps)
    # The same shots decided from the 256 initial configurations R_i L_P alone
    # (no annealing), as the baseline the annealing is compared with.
    if not args.no_greedy_only:
        fails0 = [0] * len(PS)
        for ci, c in enumerate(cases):
            sched0 = X.Schedule(c["noise"], 0, BETA0, BETA1)
            for k in range(args.warmup, n_steps):
                s0 = k * S
                X.greedy_init(code, c["noise"], c["seed"], c["shot_base"] + s0, c["syn"][s0:s0 + S], RESTARTS,
                              init=init, cbits=cbits, stream=stream)
                X.anneal(code, sched0, c["seed"], c["shot_base"] + s0, init, want_cfg=False, best_E=chain_E,
                         stream=stream)
                r0 = X.decode_reduce(code, init, cbits, chain_E, true_errors=c["err"][s0:s0 + S], stream=stream)
                fails0[ci] += int(r0["fail"].sum())
        if world > 1:
            fails0 = [int(f) for f in sum_over_ranks([float(f) for f in fails0], dist, dev)]
        if rank == 0:
            result["logical_error_rates_greedy_only"] = [stats.ler_record(p, f, S * args.steps * world)
                                                         for p, f in zip(PS, fails0)]
        # Context for the schedule: the last step's shots decoded again with the
        # annealing starting at 0.9 beta_N (the start of the paper's own
        # schedule) instead of 0.05, same 1000 sweeps and end point.
        fails9 = [0] * len(PS)
        k = n_steps - 1
        for ci, c in enumerate(cases):
            sched9 = X.Schedule(c["noise"], SWEEPS, 0.9, BETA1)
            s0 = k * S
            X.greedy_init(code, c["noise"], c["seed"], c["shot_base"] + s0, c["syn"][s0:s0 + S], RESTARTS,
                          init=init, cbits=cbits, stream=stream)
            X.anneal(code, sched9, c["seed"], c["shot_base"] + s0, init, want_cfg=False, best_E=chain_E,
                     stream=stream)
            r9 = X.decode_reduce(code, init, cbits, chain_E, true_errors=c["err"][s0:s0 + S], stream=stream)
            fails9[ci] += int(r9["fail"].sum())
        if world > 1:
            fails9 = [int(f) for f in sum_over_ranks([float(f) for f in fails9], dist, dev)]
        if rank == 0:
            result["logical_error_rates_beta0_0.9"] = [stats.ler_record(p, f, S * world) for p, f in zip(PS, fails9)]
    # ---------------------------------------------------------------- oracle parity (rank 0)
    if rank == 0 and parity.pool is not None:
        result["parity"] = parity.compare(last_outs, code.words)
    # ---------------------------------------------------------------- e2e through the C ABI, host buffers
    # Every step copies its own shots' syndromes and true errors in from
    # pinned host memory, decodes them with xzzx_decode_batch, and copies the
    # classes and failure flags out; steps take fresh shots.
    if not args.no_e2e:
        c = cases[2]
        syn_h = c["syn"].cpu().pin_memory()
        err_h = c["err"].cpu().pin_memory()
        syn_d = torch.empty_like(c["syn"][:S])
        err_d = torch.empty_like(c["err"][:S])
        cls_h = torch.empty(S, dtype=torch.uint8).pin_memory()
        fail_h = torch.empty(S, dtype=torch.uint8).pin_memory()
        ws = torch.empty(X.decode_workspace_size(code, S, RESTARTS), dtype=torch.uint8, device=dev)
        o = {k: v for k, v in outs[2]["res"].items()}

        def e2e_step(k):
            s0 = (k % n_steps) * S
            syn_d.copy_(syn_h[s0:s0 + S], non_blocking=True)
            err_d.copy_(err_h[s0:s0 + S], non_blocking=True)
            X.decode_batch(code, c["noise"], c["sched"], c["seed"], c["shot_base"] + s0, syn_d, RESTARTS,
                           true_errors=err_d, out=o, workspace=ws, stream=stream)
            cls_h.copy_(o["cls"], non_blocking=True)
            fail_h.copy_(o["fail"], non_blocking=True)
            torch.cuda.current_stream().synchronize()

        for k in range(min(args.warmup, 1)):
            e2e_step(k)
        barrier()
        t0 = time.perf_counter()
        n_e2e = args.steps
        for k in range(n_e2e):
            e2e_step(args.warmup + k)
        barrier()
        e2e_s = (time.perf_counter() - t0) / n_e2e
        if world > 1:
            e2e_s = max_over_ranks([e2e_s], dist, dev)[0]
        if rank == 0:
            result["e2e"] = {"value": S * attempts_per_shot() * world / e2e_s, "unit": "move-attempts/s",
                             "h2d_bytes_per_step": S * (syn_h.shape[1] + err_h.shape[1]) * 4,
                             "d2h_bytes_per_step": cls_h.numel() + fail_h.numel(),
                             "shots_per_s": S * world / e2e_s, "steps": n_e2e,
                             "note": "per step one batch of %d fresh shots at p=0.16 through xzzx_decode_batch: "
                                     "pinned host syndromes and true errors copied in, classes and failure "
                                     "flags copied out, stream synchronised" % S}
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args.cpu_shots)
        result["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.cpu_shots_per_core)
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
