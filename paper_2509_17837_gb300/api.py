"""Python binding of libxzzx (argument marshalling only).

The functions mirror the C entry points of ``include/xzzx.h`` one to one.
Device buffers are torch CUDA tensors (int32 or uint8 storage holding the
words and bytes of the C layout); every step of the decoder runs in the CUDA
kernels of libxzzx.  Optional output tensors are allocated with torch on the
current device when not given.
"""
import ctypes as C

import torch

from ._lib import (XZZX_ETIMEOUT, BatchCfg, BatchInfo, CodeInfo, Noise, Result, Segment, ServeCfg, ServeStats,
                   XzzxError, call, lib)

LINEAR, PAPER_LOG = 0, 1
CONVENTION_Y_OVER_XZ, CONVENTION_PAPER = 0, 1
LAYOUT_ROTATED, LAYOUT_PLANAR = 0, 1         # xzzx_make_code layouts
ORDER_COLOUR, ORDER_RANDOM_SITE = 0, 1       # sweep order of xzzx_anneal_variant
EMIN_PER_PHASE, EMIN_PER_ATTEMPT = 0, 1      # when the minimum is taken


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def version():
    return lib().xzzx_version().decode()


class Code:
    """Distance-d XZZX code (Sec. "The XZZX code"): the rotated lattice
    (layout 0) or the paper's planar lattice (layout 1); tables on the current
    GPU."""

    def __init__(self, d, layout=LAYOUT_ROTATED):
        h = C.c_void_p()
        call("xzzx_make_code", d, layout, C.byref(h))
        self._h = h
        info = CodeInfo()
        call("xzzx_get_code_info", h, C.byref(info))
        self.d = info.d
        self.layout = layout
        self.n_qubits = info.n_qubits
        self.n_stab = info.n_stab
        self.words = info.words
        self.syn_words = info.syn_words
        self.colour_start = list(info.colour_start)

    @property
    def handle(self):
        return self._h

    def faces(self):
        import numpy as np
        a = np.zeros(self.n_stab, np.int32)
        b = np.zeros(self.n_stab, np.int32)
        corners = np.zeros((self.n_stab, 4), np.int32)
        call("xzzx_code_faces", self._h, a.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p),
             corners.ctypes.data_as(C.c_void_p))
        return a, b, corners

    def device_errors(self, clear=False, stream=None):
        """(flags, count) of the device-side errors raised by work done with
        this code (XZZX_DEVERR_*); synchronises the stream."""
        flags, count = C.c_uint32(), C.c_uint32()
        call("xzzx_device_errors", self._h, C.byref(flags), C.byref(count), int(bool(clear)), _stream(stream))
        return flags.value, count.value

    def debug_inject(self, flags, stream=None):
        """Test hook: make the kernels raise these XZZX_DEVERR_* flags."""
        call("xzzx_debug_inject", self._h, flags, _stream(stream))

    def close(self):
        if self._h:
            lib().xzzx_free_code(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_noise(px, py, pz, scale=1024):
    n = Noise()
    call("xzzx_make_noise", px, py, pz, scale, C.byref(n))
    return n


def noise_from_eta(p, eta, convention=CONVENTION_Y_OVER_XZ, scale=1024):
    n = Noise()
    call("xzzx_noise_from_eta", p, eta, convention, scale, C.byref(n))
    return n


class Schedule:
    """FP64 acceptance-threshold table of an annealing schedule, uploaded once."""

    def __init__(self, noise, n_sweeps, beta0, beta1, kind=LINEAR):
        h = C.c_void_p()
        call("xzzx_make_schedule", C.byref(noise), kind, n_sweeps, beta0, beta1, C.byref(h))
        self._h = h
        self.noise = noise
        self.n_sweeps = n_sweeps

    @property
    def handle(self):
        return self._h

    def table(self):
        import numpy as np
        k = C.c_int()
        call("xzzx_schedule_table", self._h, C.byref(k), None, 0, None)
        dE = np.zeros(k.value, np.int32)
        T = np.zeros((self.n_sweeps, k.value), np.uint32)
        call("xzzx_schedule_table", self._h, C.byref(k), dE.ctypes.data_as(C.c_void_p), k.value,
             T.ctypes.data_as(C.c_void_p))
        return dE, T

    def close(self):
        if self._h:
            lib().xzzx_free_schedule(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _empty(shape, dtype, device=None):
    return torch.empty(shape, dtype=dtype, device=device if device is not None else torch.cuda.current_device())


def sample_errors(code, noise, seed, shot0, n_shots, errors=None, syndromes=None, want_errors=True, stream=None):
    if want_errors and errors is None:
        errors = _empty((n_shots, 2 * code.words), torch.int32)
    if syndromes is None:
        syndromes = _empty((n_shots, code.syn_words), torch.int32)
    call("xzzx_sample_errors", code.handle, C.byref(noise), seed, shot0, n_shots, _ptr(errors), _ptr(syndromes),
         _stream(stream))
    return errors, syndromes


def greedy_init(code, noise, seed, shot0, syndromes, restarts, randomised=True, init=None, cbits=None,
                stream=None):
    n = syndromes.shape[0]
    if init is None:
        init = _empty((n, restarts, 2 * code.words), torch.int32)
    if cbits is None:
        cbits = _empty((n, restarts), torch.uint8)
    call("xzzx_greedy_init", code.handle, C.byref(noise), seed, shot0, n, restarts, int(randomised),
         _ptr(syndromes), _ptr(init), _ptr(cbits), _stream(stream))
    return init, cbits


def anneal(code, sched, seed, shot0, init, want_cfg=True, want_final=False, best_E=None, best_cfg=None,
           final_E=None, final_cfg=None, stream=None, per_warp=False, order=ORDER_COLOUR, emin=EMIN_PER_PHASE):
    """Alg. 2 for every chain.  per_warp selects xzzx_anneal_warp; a non-default
    order (ORDER_RANDOM_SITE) or emin (EMIN_PER_ATTEMPT) selects
    xzzx_anneal_variant, the literal forms of Alg. 2 / Alg. 3."""
    n, restarts = init.shape[0], init.shape[1]
    chains = n * restarts * 4
    if best_E is None:
        best_E = _empty((n, restarts, 4), torch.int32)
    if want_cfg and best_cfg is None:
        best_cfg = _empty((n, restarts, 4, 2 * code.words), torch.int32)
    if want_final:
        final_E = final_E if final_E is not None else _empty((n, restarts, 4), torch.int32)
        final_cfg = final_cfg if final_cfg is not None else _empty((n, restarts, 4, 2 * code.words), torch.int32)
    assert best_E.numel() == chains
    if order != ORDER_COLOUR or emin != EMIN_PER_PHASE:
        if per_warp:
            raise ValueError("the warp-per-chain kernel runs the colour sweep with per-phase minima only")
        call("xzzx_anneal_variant", code.handle, sched.handle, seed, shot0, n, restarts, int(order), int(emin),
             _ptr(init), _ptr(best_E), _ptr(best_cfg), _ptr(final_E), _ptr(final_cfg), _stream(stream))
    else:
        call("xzzx_anneal_warp" if per_warp else "xzzx_anneal", code.handle, sched.handle, seed, shot0, n, restarts,
             _ptr(init), _ptr(best_E),
             _ptr(best_cfg), _ptr(final_E), _ptr(final_cfg), _stream(stream))
    return dict(best_E=best_E, best_cfg=best_cfg, final_E=final_E, final_cfg=final_cfg)


def decode_reduce(code, init, cbits, chain_E, chain_cfg=None, true_errors=None, want_best_cfg=False, stream=None):
    n, restarts = init.shape[0], init.shape[1]
    cls = _empty((n,), torch.uint8)
    E4 = _empty((n, 4), torch.int32)
    recovery = _empty((n, 2 * code.words), torch.int32)
    best = _empty((n, 2 * code.words), torch.int32) if want_best_cfg else None
    fail = _empty((n,), torch.uint8) if true_errors is not None else None
    call("xzzx_decode_reduce", code.handle, n, restarts, _ptr(init), _ptr(cbits), _ptr(chain_E), _ptr(chain_cfg),
         _ptr(true_errors), _ptr(cls), _ptr(E4), _ptr(recovery), _ptr(best), _ptr(fail), _stream(stream))
    return dict(cls=cls, E4=E4, recovery=recovery, best_cfg=best, fail=fail)


def decode_workspace_size(code, n_shots, restarts, want_best_cfg=False):
    b = C.c_size_t()
    call("xzzx_decode_workspace_size", code.handle, n_shots, restarts, int(bool(want_best_cfg)), C.byref(b))
    return b.value


def decode_batch(code, noise, sched, seed, shot0, syndromes, restarts, randomised=True, true_errors=None,
                 want_best_cfg=False, out=None, workspace=None, stream=None):
    """Alg. 7 for a batch of syndromes; returns dict(cls, E4, recovery, best_cfg, fail)."""
    n = syndromes.shape[0]
    if out is None:
        out = dict(cls=_empty((n,), torch.uint8), E4=_empty((n, 4), torch.int32),
                   recovery=_empty((n, 2 * code.words), torch.int32),
                   best_cfg=_empty((n, 2 * code.words), torch.int32) if want_best_cfg else None,
                   fail=_empty((n,), torch.uint8) if true_errors is not None else None)
    need = decode_workspace_size(code, n, restarts, want_best_cfg)
    if workspace is None or workspace.numel() < need:
        workspace = _empty((max(need, 256),), torch.uint8)
    call("xzzx_decode_batch", code.handle, C.byref(noise), sched.handle, seed, shot0, n, restarts,
         int(randomised), _ptr(syndromes), _ptr(true_errors), _ptr(out["cls"]), _ptr(out["E4"]),
         _ptr(out["recovery"]), _ptr(out.get("best_cfg")), _ptr(out.get("fail")), _ptr(workspace),
         workspace.numel(), _stream(stream))
    return out


class Batch:
    """Many homogeneous segments decoded together (xzzx_batch_*).

    segments: list of dicts with keys code, noise, sched, shot0, syndromes,
    restarts, and optionally randomised (default True) and true_errors.
    Output tensors (cls, E4, recovery, fail) are allocated per segment and
    exposed as ``self.outputs``.  run(mode): 0 = one persistent launch,
    1 = one launch per distance, 2 = as 1 with one warp per chain, 3 = the
    distances' own launches concurrently on forked streams, 4 = one
    persistent launch per distance class concurrently on forked streams.
    run_graph replays graph_mode (0, 3 or 4) as a captured CUDA graph.
    """

    def __init__(self, segments, seed, ctas_per_sm=0, order=0, graph_mode=0, chains_per_cta=0, sweep_unroll=0):
        self.segments = segments
        self.outputs = []
        arr = (Segment * len(segments))()
        self._keep = []
        for j, sg in enumerate(segments):
            code, syn = sg["code"], sg["syndromes"]
            n = syn.shape[0]
            err = sg.get("true_errors")
            out = dict(cls=_empty((n,), torch.uint8), E4=_empty((n, 4), torch.int32),
                       recovery=_empty((n, 2 * code.words), torch.int32),
                       fail=_empty((n,), torch.uint8) if err is not None else None)
            self.outputs.append(out)
            a = arr[j]
            a.code, a.noise, a.sched = code.handle, C.addressof(sg["noise"]), sg["sched"].handle
            a.shot0, a.n_shots, a.restarts = sg.get("shot0", 0), n, sg["restarts"]
            a.randomised = int(sg.get("randomised", 1))
            a.syndromes = syn.data_ptr() if n else None
            a.true_errors = err.data_ptr() if err is not None and n else None
            a.cls = out["cls"].data_ptr() if n else None
            a.E4 = out["E4"].data_ptr() if n else None
            a.recovery = out["recovery"].data_ptr() if n else None
            a.fail = out["fail"].data_ptr() if out["fail"] is not None and n else None
        cfg = BatchCfg(ctas_per_sm, order, graph_mode, chains_per_cta, sweep_unroll)
        h = C.c_void_p()
        call("xzzx_batch_create", arr, len(segments), seed, C.byref(cfg), C.byref(h))
        self._h = h

    def run(self, mode=0, stream=None):
        call("xzzx_batch_run", self._h, mode, _stream(stream))

    def run_graph(self, stream):
        call("xzzx_batch_run_graph", self._h, C.c_void_p(stream.cuda_stream))

    def info(self):
        i = BatchInfo()
        call("xzzx_batch_get_info", self._h, C.byref(i))
        return {k: getattr(i, k) for k, _ in BatchInfo._fields_}

    def close(self):
        if self._h:
            lib().xzzx_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Decode server with continuous batching (xzzx_serve_*).

    Requests are single syndromes (host uint32 words) of registered
    (distance, noise) classes; results come back with their latency.
    """

    def __init__(self, seed, restarts, n_sweeps, beta0, beta1, kind=LINEAR, max_batch=256, n_slots=4,
                 queue_capacity=1 << 20, hbm_budget_bytes=0, warp_max_requests=0, resident_waves=0):
        cfg = ServeCfg(seed, restarts, n_sweeps, kind, beta0, beta1, max_batch, n_slots, queue_capacity,
                       hbm_budget_bytes, warp_max_requests, resident_waves)
        h = C.c_void_p()
        call("xzzx_serve_create", C.byref(cfg), C.byref(h))
        self._h = h
        self.classes = []

    def add_class(self, d, noise):
        cid = C.c_int()
        call("xzzx_serve_add_class", self._h, d, C.byref(noise), C.byref(cid))
        self.classes.append((d, noise))
        return cid.value

    def start(self):
        call("xzzx_serve_start", self._h)

    def submit(self, req_id, class_id, syndrome_words):
        import numpy as np
        w = np.ascontiguousarray(syndrome_words, dtype=np.uint32)
        return lib().xzzx_serve_submit(self._h, req_id, class_id, w.ctypes.data_as(C.c_void_p))

    def replay(self, req_ids, class_ids, syndromes32, arrival_us):
        import numpy as np
        ids = np.ascontiguousarray(req_ids, dtype=np.uint64)
        cls = np.ascontiguousarray(class_ids, dtype=np.int32)
        syn = np.ascontiguousarray(syndromes32, dtype=np.uint32)
        at = np.ascontiguousarray(arrival_us, dtype=np.float64)
        assert syn.shape == (len(ids), 32)
        call("xzzx_serve_replay", self._h, len(ids), ids.ctypes.data_as(C.c_void_p), cls.ctypes.data_as(C.c_void_p),
             syn.ctypes.data_as(C.c_void_p), at.ctypes.data_as(C.c_void_p))

    def poll(self, cap=4096, timeout_ms=100):
        buf = (Result * cap)()
        n = C.c_int()
        st = lib().xzzx_serve_poll(self._h, buf, cap, C.byref(n), timeout_ms)
        if st not in (0, XZZX_ETIMEOUT):
            raise XzzxError(st, "xzzx_serve_poll", lib().xzzx_last_error().decode())
        out = []
        for i in range(n.value):
            r = buf[i]
            w = (r.d * r.d + 31) // 32
            out.append(dict(req_id=r.req_id, class_id=r.class_id, d=r.d, cls=r.cls, E4=list(r.E4),
                            recovery=list(r.recovery[:2 * w]), latency_us=r.latency_us))
        return out

    def stats(self, reset=False):
        st = ServeStats()
        call("xzzx_serve_get_stats", self._h, C.byref(st), int(bool(reset)))
        return {k: getattr(st, k) for k, _ in ServeStats._fields_}

    def close(self):
        if self._h:
            lib().xzzx_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
