"""The FP32 GEMM of the mixed form (include/gev_kernels.h): BF16 split products on the tensor cores
(tcgen05; engine 1 = BF16x6, engine 2 = BF16x3) and the FP32 CUDA-core engine (0), against an
FP64 product of the same FP32 operands.

Error bounds from the arithmetic: the three-way BF16 split is exact for FP32 values and BF16x6 drops
only the pairs with p + q >= 5 (below 2^-24 of each product), so with FP32 accumulation over K
terms it stays below 1e-5 (|A| |B|)_ij for the K used here, like the FP32 engine; BF16x3 keeps about
16 bits per product: below 1e-4 (|A| |B|)_ij."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (128, 128, 64), (200, 130, 300), (257, 513, 1000), (1024, 768, 2048), (96, 100, 5000),
          (700, 64, 3000), (50, 700, 2000), (300, 33, 700)]


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2502_02460_gb300 import build, gev

    build.build()
    L = gev.lib()
    vp, i = ctypes.c_void_p, ctypes.c_int
    L.gev_gemm_f32.argtypes = [i, i, i, i, i, ctypes.c_float, vp, i, vp, i, ctypes.c_float, vp, i, i, vp, vp, vp,
                               ctypes.c_size_t]
    L.gev_gemm_f32.restype = i
    L.gev_gemm_f32_scratch_bytes.argtypes = [i, i, i]
    L.gev_gemm_f32_scratch_bytes.restype = ctypes.c_size_t
    return L, torch, torch.device("cuda:0")


@pytest.mark.parametrize("engine", [1, 2, 0])
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_gemm_f32_matches_fp64(env, engine, ta, tb, M, N, K):
    L, torch, dev = env
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K + 11 * ta + 5 * tb)
    opA = torch.randn(M, K, generator=g, dtype=torch.float64)
    opB = torch.randn(K, N, generator=g, dtype=torch.float64)
    C0 = torch.randn(M, N, generator=g, dtype=torch.float64)
    alpha, beta = 0.75, -0.5
    # column-major device buffers: a (rows x cols) column-major matrix is the row-major buffer of its
    # transpose
    Astore = opA if ta == 0 else opA.T  # stored matrix (column-major)
    Bstore = opB if tb == 0 else opB.T
    Ab = Astore.T.contiguous().float().to(dev)
    Bb = Bstore.T.contiguous().float().to(dev)
    Cb = C0.T.contiguous().float().to(dev)
    st = torch.zeros(16, dtype=torch.int32, device=dev)
    lda, ldb = Astore.shape[0], Bstore.shape[0]
    stream = torch.cuda.current_stream(dev)
    nbytes = L.gev_gemm_f32_scratch_bytes(M, N, K)
    scr = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    code = L.gev_gemm_f32(M, N, K, ta, tb, alpha, ctypes.c_void_p(Ab.data_ptr()), lda,
                          ctypes.c_void_p(Bb.data_ptr()), ldb, beta, ctypes.c_void_p(Cb.data_ptr()), M,
                          engine, ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(st.data_ptr()),
                          ctypes.c_void_p(scr.data_ptr()), nbytes)
    assert code == 0
    assert int(st[1].item()) == 0
    C = Cb.cpu().double().T
    # reference from the FP32-rounded inputs, in FP64
    Ar = Astore.float().double()
    Br = Bstore.float().double()
    opAr = Ar if ta == 0 else Ar.T
    opBr = Br if tb == 0 else Br.T
    ref = alpha * (opAr @ opBr) + beta * C0.float().double()
    scale = abs(alpha) * (opAr.abs() @ opBr.abs()) + abs(beta) * C0.abs()
    tol = 1e-4 if engine == 2 else 1e-5
    err = ((C - ref).abs() / scale.clamp_min(1e-30)).max().item()
    assert err <= tol, err
