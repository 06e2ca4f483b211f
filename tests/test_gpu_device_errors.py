"""Device-side failures surface on the host instead of being dropped.

Kernels never trap: a failure they detect is recorded in the error area of the
code handle the work used (xzzx_device_errors reads it).  Failures are made on
the host side only: xzzx_debug_inject asks the kernels to take their own
failure path as if the failure had happened, so no GPU fault is ever caused.

* A greedy walk failure (XZZX_DEVERR_GREEDY_WALK) sets bit 7 of the restart's
  class byte and the code's error flags, through xzzx_greedy_init, the fused
  decoder and the batch path; a clean run leaves the flags at zero.
* The checked build (-DXZZX_CHECKS, libxzzx_checks.so) gives bit-identical
  results to the plain build with no flag raised, and its annealing bounds
  check records XZZX_DEVERR_BOUNDS when made to fail.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2509_17837_gb300 import build
    build.build()
    import torch

    import paper_2509_17837_gb300 as X
    return X, torch


def test_clean_decode_raises_nothing(env):
    X, torch = env
    code = X.Code(11)
    noise = X.noise_from_eta(0.16, 100)
    sched = X.Schedule(noise, 50, 0.05, 20.0)
    err, syn = X.sample_errors(code, noise, 7, 0, 500)
    X.decode_batch(code, noise, sched, 7, 0, syn, 16, true_errors=err)
    assert code.device_errors() == (0, 0)


def test_injected_greedy_walk_failure_is_reported(env):
    X, torch = env
    from paper_2509_17837_gb300._lib import XZZX_DEVERR_GREEDY_WALK
    d, n, R = 9, 37, 6
    code = X.Code(d)
    noise = X.noise_from_eta(0.15, 10)
    err, syn = X.sample_errors(code, noise, 3, 0, n)
    ref_init, ref_cb = X.greedy_init(code, noise, 3, 0, syn, R)
    code.debug_inject(XZZX_DEVERR_GREEDY_WALK)
    init, cb = X.greedy_init(code, noise, 3, 0, syn, R)
    flags, count = code.device_errors(clear=True)
    assert flags == XZZX_DEVERR_GREEDY_WALK and count == n
    cb_h, ref_h = cb.cpu().numpy(), ref_cb.cpu().numpy()
    assert (cb_h[:, 0] & 0x80).all() and not (cb_h[:, 1:] & 0x80).any()
    assert np.array_equal(cb_h & 0x7F, ref_h) and torch.equal(init, ref_init)   # references unchanged
    # through the fused decoder and the batch path too
    sched = X.Schedule(noise, 20, 0.05, 20.0)
    X.decode_batch(code, noise, sched, 3, 0, syn, R, true_errors=err)
    assert code.device_errors(clear=True) == (XZZX_DEVERR_GREEDY_WALK, n)
    b = X.Batch([dict(code=code, noise=noise, sched=sched, shot0=0, syndromes=syn, restarts=R, true_errors=err)], 3)
    b.run(0)
    assert code.device_errors(clear=True) == (XZZX_DEVERR_GREEDY_WALK, n)
    code.debug_inject(0)
    X.decode_batch(code, noise, sched, 3, 0, syn, R, true_errors=err)
    assert code.device_errors() == (0, 0)


def test_server_reports_no_device_errors_on_clean_work(env):
    X, torch = env
    sv = X.Server(11, 4, 30, 0.05, 20.0, max_batch=8, n_slots=2)
    try:
        cid = sv.add_class(5, X.noise_from_eta(0.1, 10))
        sv.start()
        code = X.Code(5)
        _, syn = X.sample_errors(code, X.noise_from_eta(0.1, 10), 11, 0, 20, want_errors=False)
        words = np.zeros((20, 32), np.uint32)
        words[:, :code.syn_words] = syn.cpu().numpy().view(np.uint32)
        for k in range(20):
            assert sv.submit(k, cid, words[k]) == 0
        got = 0
        for _ in range(200):
            got += len(sv.poll(timeout_ms=100))
            if got == 20:
                break
        assert got == 20
        assert sv.stats()["device_errors"] == 0
    finally:
        sv.close()


def _checked_lib():
    from paper_2509_17837_gb300 import build
    from paper_2509_17837_gb300._lib import SIGNATURES
    L = ctypes.CDLL(build.build(checks=True))
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


def test_checked_build_matches_and_reports_bounds(env):
    X, torch = env
    from paper_2509_17837_gb300._lib import XZZX_DEVERR_BOUNDS, XZZX_OK, Noise
    L = _checked_lib()
    d, n, R, N, seed = 11, 200, 16, 100, 0xC4EC
    noise = X.noise_from_eta(0.16, 100)
    code, sched = X.Code(d), X.Schedule(noise, N, 0.05, 20.0)
    err, syn = X.sample_errors(code, noise, seed, 0, n)
    ref = X.decode_batch(code, noise, sched, seed, 0, syn, R, true_errors=err, want_best_cfg=True)
    torch.cuda.synchronize()

    def ok(st):
        assert st == XZZX_OK, L.xzzx_last_error()

    hc, hs = ctypes.c_void_p(), ctypes.c_void_p()
    ok(L.xzzx_make_code(d, 0, ctypes.byref(hc)))
    nz = Noise()
    ok(L.xzzx_noise_from_eta(0.16, 100.0, 0, 1024, ctypes.byref(nz)))
    ok(L.xzzx_make_schedule(ctypes.byref(nz), 0, N, 0.05, 20.0, ctypes.byref(hs)))
    try:
        size = ctypes.c_size_t()
        ok(L.xzzx_decode_workspace_size(hc, n, R, 1, ctypes.byref(size)))
        ws = torch.empty(size.value, dtype=torch.uint8, device="cuda")
        got = {k: torch.empty_like(v) for k, v in ref.items() if v is not None}
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        ok(L.xzzx_decode_batch(hc, ctypes.byref(nz), hs, seed, 0, n, R, 1, p(syn), p(err), p(got["cls"]),
                               p(got["E4"]), p(got["recovery"]), p(got["best_cfg"]), p(got["fail"]), p(ws),
                               size.value, stream))
        flags, count = ctypes.c_uint32(), ctypes.c_uint32()
        ok(L.xzzx_device_errors(hc, ctypes.byref(flags), ctypes.byref(count), 1, stream))
        assert (flags.value, count.value) == (0, 0)
        for k in got:
            assert torch.equal(got[k], ref[k]), k
        # make the annealing lookup's bounds check fail: recorded, nothing faults
        ok(L.xzzx_debug_inject(hc, XZZX_DEVERR_BOUNDS, stream))
        ok(L.xzzx_decode_batch(hc, ctypes.byref(nz), hs, seed, 0, 8, R, 1, p(syn), p(err), p(got["cls"]),
                               p(got["E4"]), p(got["recovery"]), p(got["best_cfg"]), p(got["fail"]), p(ws),
                               size.value, stream))
        ok(L.xzzx_device_errors(hc, ctypes.byref(flags), ctypes.byref(count), 1, stream))
        assert flags.value == XZZX_DEVERR_BOUNDS and count.value > 0
        ok(L.xzzx_debug_inject(hc, 0, stream))
    finally:
        L.xzzx_free_schedule(hs)
        L.xzzx_free_code(hc)
