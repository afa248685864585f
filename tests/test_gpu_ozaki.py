"""FP64 products formed on the BF16 tensor cores (gev_gemm_f64, engine 1) and the native FP64 DMMA
path (engine 0), against an FP64 reference (torch/cuBLAS on the same device).

Bound from the construction: the scaled digits are exact to 2^-56 of the row / column scale, the
dropped digit pairs are below 2^-56 of it, and every sum is exact except the FP64 epilogue and the
shared low-order accumulator, so |C - C_ref| <= 4e-15 (|A| |B|)_ij (about 2^-48) for the K used
here; the same bound holds for the native path."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (128, 64, 64), (130, 70, 200), (257, 513, 1000), (1024, 512, 4096)]


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2502_02460_gb300 import build, gev

    build.build()
    L = gev.lib()
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.gev_gemm_f64.argtypes = [i, i, i, i, i, d, vp, i, vp, i, d, vp, i, i, vp, vp, vp]
    L.gev_gemm_f64.restype = i
    return L, torch, torch.device("cuda:0")


def run(env, M, N, K, ta, tb, engine, scale_rows=False, seed=0):
    L, torch, dev = env
    g = torch.Generator().manual_seed(seed + M + 3 * N + 7 * K)
    opA = torch.randn(M, K, generator=g, dtype=torch.float64)
    opB = torch.randn(K, N, generator=g, dtype=torch.float64)
    if scale_rows:  # wide dynamic range across rows and columns
        opA *= torch.logspace(-8, 8, M, dtype=torch.float64)[:, None]
        opB *= torch.logspace(6, -6, N, dtype=torch.float64)[None, :]
    C0 = torch.randn(M, N, generator=g, dtype=torch.float64)
    alpha, beta = 1.25, -0.75
    Astore = opA if ta == 0 else opA.T
    Bstore = opB if tb == 0 else opB.T
    Ab, Bb, Cb = (x.T.contiguous().to(dev) for x in (Astore, Bstore, C0))
    st = torch.zeros(16, dtype=torch.int32, device=dev)
    scr = torch.zeros(2 * (max(M, N) + 8), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    code = L.gev_gemm_f64(M, N, K, ta, tb, alpha, ctypes.c_void_p(Ab.data_ptr()), Astore.shape[0],
                          ctypes.c_void_p(Bb.data_ptr()), Bstore.shape[0], beta, ctypes.c_void_p(Cb.data_ptr()),
                          M, engine, ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(st.data_ptr()),
                          ctypes.c_void_p(scr.data_ptr()))
    assert code == 0 and int(st[1].item()) == 0
    C = Cb.cpu().T
    ref = alpha * (opA.to(dev) @ opB.to(dev)).cpu() + beta * C0
    scale = abs(alpha) * (opA.abs() @ opB.abs()) + abs(beta) * C0.abs()
    return ((C - ref).abs() / scale.clamp_min(1e-300)).max().item()


@pytest.mark.parametrize("engine", [1, 0])
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_gemm_f64_engines(env, engine, ta, tb, M, N, K):
    assert run(env, M, N, K, ta, tb, engine) <= 4e-15


@pytest.mark.parametrize("engine", [1, 0])
def test_gemm_f64_wide_dynamic_range(env, engine):
    assert run(env, 300, 200, 700, 0, 1, engine, scale_rows=True) <= 4e-15
