"""The no-allocation Cholesky entry point gev_potrf_noalloc (include/gev_noalloc.h).

Some callers of this library cannot call cudaMalloc: their device memory belongs to another memory
manager (a caching allocator or pool with a fixed budget), or an allocation's implicit
synchronisation is not acceptable in their loop.  gev_potrf_noalloc serves them from a fixed scratch
array compiled into the library.  This test calls it through the C ABI and checks it against the
handle-based entry point gev_step_potrf on two calls in a row (the second call reuses the same
scratch); it also checks the size limit.  The file name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest

from paper_2502_02460_gb300 import inputs

pytestmark = pytest.mark.gpu

MAX_N = 4096
ERR_TOO_LARGE = 8


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2502_02460_gb300 import build, gev

    build.build()
    L = gev.lib()
    L.gev_potrf_noalloc.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_int)]
    L.gev_potrf_noalloc.restype = ctypes.c_int
    assert torch.cuda.is_available()
    return L, gev, torch.device("cuda:0")


def noalloc(L, buf, n, stream):
    info = ctypes.c_int(-7)
    code = L.gev_potrf_noalloc(n, ctypes.c_void_p(buf.data_ptr()), n,
                               ctypes.c_void_p(stream.cuda_stream), ctypes.byref(info))
    return code, info.value


def reference(gev, S, dev):
    n = S.shape[0]
    with gev.Solver(n, device=dev) as s:
        B = gev.cm_from_numpy(S, dev)
        assert s.potrf(B) == 0
        return gev.numpy_from_cm(B)


def test_noalloc_cholesky_matches_handle_entry_on_two_calls(env):
    import torch

    L, gev, dev = env
    stream = torch.cuda.current_stream(dev)
    eps = np.finfo(np.float64).eps
    for n, seed in ((777, 1), (300, 2)):  # two calls in a row: the second reuses the scratch
        S = inputs.make_problem(n, 1, seed=seed).S
        ref = reference(gev, S, dev)
        buf = gev.cm_from_numpy(inputs.lower_only(S, 5.0), dev)
        code, info = noalloc(L, buf, n, stream)
        assert code == 0 and info == 0
        got = gev.numpy_from_cm(buf)
        assert np.max(np.abs(got - ref)) <= 64 * n * eps * np.abs(ref).max()
        assert np.all(np.triu(got, 1) == 0)


def test_noalloc_rejects_sizes_beyond_the_scratch_and_reports_pivots(env):
    import torch

    L, gev, dev = env
    stream = torch.cuda.current_stream(dev)
    big = torch.zeros((8, 8), dtype=torch.float64, device=dev)  # never touched: rejected first
    info = ctypes.c_int(0)
    assert L.gev_potrf_noalloc(MAX_N + 1, ctypes.c_void_p(big.data_ptr()), MAX_N + 1,
                               ctypes.c_void_p(stream.cuda_stream), ctypes.byref(info)) == ERR_TOO_LARGE
    S = np.eye(200)
    S[150, 150] = -1.0
    code, info = noalloc(L, gev.cm_from_numpy(S, dev), 200, stream)
    assert code == 1 and info == 151
