"""The no-allocation Cholesky entry point gev_potrf_noalloc (include/gev_noalloc.h).

Some callers of this library cannot call cudaMalloc: their device memory belongs to another memory
manager (a caching allocator or pool with a fixed budget), or an allocation's implicit
synchronisation is not acceptable in their loop.  gev_potrf_noalloc serves them from a fixed scratch
array compiled into the library.  This test calls it through the C ABI and checks it, on two calls in
a row (the second reuses the same scratch), against the FP64 CPU oracle's Cholesky factor and against
the handle-based entry point gev_step_potrf on a handle with native FP64 products (the same kernels:
bit for bit); it checks that a call changes the device's free memory by nothing, and the size limit.
The file name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest

import oracle
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


def handle_factor(gev, S, dev):
    """gev_step_potrf on a handle whose products run on native FP64 (DMMA), as the no-allocation
    path's do (the emulated products need workspace that a handle allocates)."""
    n = S.shape[0]
    with gev.Solver(n, device=dev, fp64_emulation=0) as s:
        B = gev.cm_from_numpy(S, dev)
        assert s.potrf(B) == 0
        return gev.numpy_from_cm(B)


def test_noalloc_cholesky_matches_oracle_and_handle_entry_on_two_calls(env):
    import torch

    L, gev, dev = env
    stream = torch.cuda.current_stream(dev)
    eps = np.finfo(np.float64).eps
    for n, seed in ((777, 1), (300, 2)):  # two calls in a row: the second reuses the scratch
        S = inputs.make_problem(n, 1, seed=seed).S
        buf = gev.cm_from_numpy(inputs.lower_only(S, 5.0), dev)
        code, info = noalloc(L, buf, n, stream)
        assert code == 0 and info == 0
        got = gev.numpy_from_cm(buf)
        assert np.all(np.triu(got, 1) == 0)
        Lo, oinfo = oracle.potrf(S)
        assert oinfo == 0
        Lo = np.tril(Lo)
        assert np.max(np.abs(got - Lo)) <= 64 * n * eps * np.abs(Lo).max()
        assert np.array_equal(got, handle_factor(gev, S, dev))


def test_noalloc_call_allocates_no_device_memory(env):
    import torch

    L, gev, dev = env
    stream = torch.cuda.current_stream(dev)
    n = MAX_N  # the largest size: the widest products of the path
    S = inputs.overlap_toeplitz(n, False)
    buf = gev.cm_from_numpy(S, dev)
    assert noalloc(L, buf.clone(), n, stream)[0] == 0  # warm: every kernel of the path is loaded
    work = buf.clone()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    code, info = noalloc(L, work, n, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert code == 0 and info == 0
    assert free1 == free0


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
