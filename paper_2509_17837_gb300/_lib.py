"""ctypes declarations of libxzzx.so (argument marshalling only).

Every function here is the C entry point of the same name in
``include/xzzx.h``; nothing is computed in Python.  Importing this module
fails loudly when the library has not been built: there is no fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libxzzx.so")

XZZX_OK, XZZX_EINVAL, XZZX_ENOMEM, XZZX_ECUDA, XZZX_ETIMEOUT, XZZX_EBUSY, XZZX_EUNSUPPORTED = range(7)
XZZX_DEVERR_GREEDY_WALK, XZZX_DEVERR_BOUNDS = 0x1, 0x2
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ETIMEOUT", "EBUSY", "EUNSUPPORTED"]


class XzzxError(RuntimeError):
    def __init__(self, status, func, msg):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s failed with XZZX_%s: %s" % (func, name, msg))


class Noise(C.Structure):
    _fields_ = [("px", C.c_double), ("py", C.c_double), ("pz", C.c_double), ("scale", C.c_int32),
                ("W", C.c_int32 * 4), ("Wt_x", C.c_int32), ("Wt_z", C.c_int32)]


class CodeInfo(C.Structure):
    _fields_ = [("d", C.c_int32), ("n_qubits", C.c_int32), ("n_stab", C.c_int32), ("words", C.c_int32),
                ("syn_words", C.c_int32), ("colour_start", C.c_int32 * 5)]


class Segment(C.Structure):
    _fields_ = [("code", C.c_void_p), ("noise", C.c_void_p), ("sched", C.c_void_p), ("shot0", C.c_uint64),
                ("n_shots", C.c_int32), ("restarts", C.c_int32), ("randomised", C.c_int32),
                ("syndromes", C.c_void_p), ("true_errors", C.c_void_p), ("cls", C.c_void_p), ("E4", C.c_void_p),
                ("recovery", C.c_void_p), ("fail", C.c_void_p)]


class BatchCfg(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int32), ("order", C.c_int32), ("graph_mode", C.c_int32),
                ("chains_per_cta", C.c_int32), ("sweep_unroll", C.c_int32)]


class BatchInfo(C.Structure):
    _fields_ = [("n_segments", C.c_int32), ("n_chunks", C.c_int32), ("n_distances", C.c_int32),
                ("persistent_grid", C.c_int32), ("launches_batched", C.c_int32), ("launches_plain", C.c_int32),
                ("workspace_bytes", C.c_size_t), ("move_attempts", C.c_double), ("total_shots", C.c_int64),
                ("chains_per_cta", C.c_int32), ("sweep_unroll", C.c_int32), ("n_classes", C.c_int32),
                ("warp_ctas_per_sm", C.c_int32)]


class ServeCfg(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("restarts", C.c_int32), ("n_sweeps", C.c_int32),
                ("sched_kind", C.c_int32), ("beta0", C.c_double), ("beta1", C.c_double),
                ("max_batch", C.c_int32), ("n_slots", C.c_int32), ("queue_capacity", C.c_int32),
                ("hbm_budget_bytes", C.c_size_t), ("warp_max_requests", C.c_int32),
                ("resident_waves", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("req_id", C.c_uint64), ("class_id", C.c_int32), ("d", C.c_int32), ("cls", C.c_int32),
                ("E4", C.c_int32 * 4), ("recovery", C.c_uint32 * 62), ("latency_us", C.c_double)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("rejected", C.c_int64), ("dispatched", C.c_int64),
                ("completed", C.c_int64), ("batches", C.c_int64), ("pending", C.c_int64),
                ("in_flight", C.c_int64), ("mean_batch", C.c_double), ("p50_us", C.c_double),
                ("p99_us", C.c_double), ("max_us", C.c_double), ("mean_us", C.c_double),
                ("device_errors", C.c_uint32)]


_p = C.c_void_p
_i = C.c_int
_u64 = C.c_uint64
_d = C.c_double

SIGNATURES = {
    "xzzx_last_error": ([], C.c_char_p),
    "xzzx_device_errors": ([_p, _p, _p, _i, _p], _i),
    "xzzx_debug_inject": ([_p, C.c_uint32, _p], _i),
    "xzzx_version": ([], C.c_char_p),
    "xzzx_abi_struct_size": ([_i], C.c_size_t),
    "xzzx_make_code": ([_i, _i, C.POINTER(_p)], _i),
    "xzzx_get_code_info": ([_p, C.POINTER(CodeInfo)], _i),
    "xzzx_free_code": ([_p], None),
    "xzzx_code_faces": ([_p, _p, _p, _p], _i),
    "xzzx_make_noise": ([_d, _d, _d, C.c_int32, C.POINTER(Noise)], _i),
    "xzzx_noise_from_eta": ([_d, _d, _i, C.c_int32, C.POINTER(Noise)], _i),
    "xzzx_make_schedule": ([C.POINTER(Noise), _i, _i, _d, _d, C.POINTER(_p)], _i),
    "xzzx_free_schedule": ([_p], None),
    "xzzx_schedule_table": ([_p, C.POINTER(_i), _p, _i, _p], _i),
    "xzzx_sample_errors": ([_p, C.POINTER(Noise), _u64, _u64, _i, _p, _p, _p], _i),
    "xzzx_greedy_init": ([_p, C.POINTER(Noise), _u64, _u64, _i, _i, _i, _p, _p, _p, _p], _i),
    "xzzx_anneal": ([_p, _p, _u64, _u64, _i, _i, _p, _p, _p, _p, _p, _p], _i),
    "xzzx_anneal_warp": ([_p, _p, _u64, _u64, _i, _i, _p, _p, _p, _p, _p, _p], _i),
    "xzzx_anneal_variant": ([_p, _p, _u64, _u64, _i, _i, _i, _i, _p, _p, _p, _p, _p, _p], _i),
    "xzzx_decode_reduce": ([_p, _i, _i, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p], _i),
    "xzzx_decode_workspace_size": ([_p, _i, _i, _i, C.POINTER(C.c_size_t)], _i),
    "xzzx_decode_batch": ([_p, C.POINTER(Noise), _p, _u64, _u64, _i, _i, _i, _p, _p, _p, _p, _p, _p, _p, _p,
                           C.c_size_t, _p], _i),
    "xzzx_batch_create": ([C.POINTER(Segment), _i, _u64, C.POINTER(BatchCfg), C.POINTER(_p)], _i),
    "xzzx_batch_run": ([_p, _i, _p], _i),
    "xzzx_batch_run_graph": ([_p, _p], _i),
    "xzzx_batch_get_info": ([_p, C.POINTER(BatchInfo)], _i),
    "xzzx_batch_destroy": ([_p], None),
    "xzzx_serve_create": ([C.POINTER(ServeCfg), C.POINTER(_p)], _i),
    "xzzx_serve_add_class": ([_p, _i, C.POINTER(Noise), C.POINTER(_i)], _i),
    "xzzx_serve_start": ([_p], _i),
    "xzzx_serve_submit": ([_p, _u64, _i, _p], _i),
    "xzzx_serve_replay": ([_p, _i, _p, _p, _p, _p], _i),
    "xzzx_serve_poll": ([_p, C.POINTER(Result), _i, C.POINTER(_i), _i], _i),
    "xzzx_serve_get_stats": ([_p, C.POINTER(ServeStats), _i], _i),
    "xzzx_serve_destroy": ([_p], None),
    "xzzx_decode_batch_static": ([_p, C.POINTER(Noise), _p, _u64, _u64, _i, _i, _i, _p, _p, _p, _p, _p, _p, _p,
                                  _p], _i),
}

_lib = None


def lib():
    """Load libxzzx.so once; raise if it is missing (no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libxzzx.so is not built (%s); run `python -c \"import __graft_entry__ as g; "
                               "g.build()\"` or `python -m paper_2509_17837_gb300.build`" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def check(status, func):
    if status != XZZX_OK:
        msg = lib().xzzx_last_error()
        raise XzzxError(status, func, msg.decode() if msg else "")


def call(name, *args):
    """Call entry point `name` and raise XzzxError on a non-OK status."""
    st = getattr(lib(), name)(*args)
    check(st, name)
    return st
