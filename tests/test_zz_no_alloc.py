"""xzzx_decode_batch_static: the allocation-free decoder entry point.

It serves callers that cannot allocate device memory while they run (a
decoder inside a control loop with a fixed GPU memory plan, or a C host that
only receives device buffers).  This test calls it through the C ABI twice in
a row, on two different batches, and checks each result bit-exactly against
xzzx_decode_batch with a caller-owned workspace (the bar all parity tests
use), after a warm-up call with no shots; around each call the device's free
memory must not change.  It then checks that an oversized batch is refused.  The file sorts last so
that a run stopping at the first failure has already run every other test.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2509_17837_gb300 import build
    build.build()
    import torch

    import paper_2509_17837_gb300 as X
    return X, torch


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def test_static_entry_point_matches_workspace_entry_point(env):
    X, torch = env
    from paper_2509_17837_gb300._lib import XZZX_OK, lib
    d, R, n = 11, 16, 300
    code = X.Code(d)
    noise = X.noise_from_eta(0.16, 100)
    sched = X.Schedule(noise, 200, 0.05, 20.0)
    assert X.decode_workspace_size(code, n, R, True) <= (16 << 20)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the start-up warm-up call: no shots, only the one-time set-up
    st = lib().xzzx_decode_batch_static(code.handle, ctypes.byref(noise), sched.handle, 1, 0, 0, R, 1, None, None,
                                        None, None, None, None, None, stream)
    assert st == XZZX_OK, lib().xzzx_last_error()
    free_before = []
    for call, (seed, shot0) in enumerate([(101, 0), (202, 5000)]):
        err, syn = X.sample_errors(code, noise, seed, shot0, n)
        ref = X.decode_batch(code, noise, sched, seed, shot0, syn, R, true_errors=err, want_best_cfg=True)
        got = dict(cls=torch.empty_like(ref["cls"]), E4=torch.empty_like(ref["E4"]),
                   recovery=torch.empty_like(ref["recovery"]), best_cfg=torch.empty_like(ref["best_cfg"]),
                   fail=torch.empty_like(ref["fail"]))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = lib().xzzx_decode_batch_static(code.handle, ctypes.byref(noise), sched.handle, seed, shot0, n, R, 1,
                                            _p(syn), _p(err), _p(got["cls"]), _p(got["E4"]), _p(got["recovery"]),
                                            _p(got["best_cfg"]), _p(got["fail"]), stream)
        assert st == XZZX_OK, lib().xzzx_last_error()
        torch.cuda.synchronize()
        free_before.append((free0, torch.cuda.mem_get_info()[0]))
        for k in ("cls", "E4", "recovery", "best_cfg", "fail"):
            assert torch.equal(got[k], ref[k]), (call, k)
    # after the warm-up no call changes the device's free memory: nothing is allocated
    for free0, free1 in free_before:
        assert free0 == free1


def test_static_entry_point_refuses_oversized_batches(env):
    X, torch = env
    from paper_2509_17837_gb300._lib import XZZX_EINVAL, lib
    code = X.Code(11)
    noise = X.noise_from_eta(0.16, 100)
    sched = X.Schedule(noise, 10, 0.05, 20.0)
    n, R = 20000, 64
    assert X.decode_workspace_size(code, n, R, False) > (16 << 20)
    syn = torch.zeros((n, code.syn_words), dtype=torch.int32, device="cuda")
    cls = torch.empty(n, dtype=torch.uint8, device="cuda")
    E4 = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    rec = torch.empty((n, 2 * code.words), dtype=torch.int32, device="cuda")
    st = lib().xzzx_decode_batch_static(code.handle, ctypes.byref(noise), sched.handle, 1, 0, n, R, 1, _p(syn), None,
                                        _p(cls), _p(E4), _p(rec), None, None, None)
    assert st == XZZX_EINVAL
    assert b"split the batch" in lib().xzzx_last_error()
