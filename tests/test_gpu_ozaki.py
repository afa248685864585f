"""FP64 products formed on the BF16 tensor cores (gev_gemm_f64, engine 1) and the native FP64 DMMA
path (engine 0), against an FP64 reference (torch/cuBLAS on the same device).

Bound from the construction: the scaled digits are exact to 2^-55 of the row / column scale, the
dropped digit pairs are below 2^-55 of it, and every sum is exact except the FP64 epilogue and the
shared low-order accumulator.  For entries of similar magnitude within each row and column, as
here (and, with the row scaling, in the wide-range test), that gives |C - C_ref| <= 4e-15
(|A| |B|)_ij (about 2^-48) for the K used here; the same bound holds for the native path.  The
general bound, relative to the row and column scales, is checked on a CPU model of the scheme in
tests/test_fp64_emulation_model.py.  The shapes cover one and several 512-deep exact
chunks, ragged tiles, split K (few output tiles, long K) and K above one launch's 32768."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (128, 64, 64), (130, 70, 200), (257, 513, 1000), (1024, 512, 4096), (96, 80, 9000)]


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2502_02460_gb300 import build, gev

    build.build()
    L = gev.lib()
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.gev_gemm_f64.argtypes = [i, i, i, i, i, d, vp, i, vp, i, d, vp, i, i, vp, vp, vp, ctypes.c_size_t]
    L.gev_gemm_f64.restype = i
    L.gev_gemm_f64_scratch_bytes.argtypes = [i, i, i]
    L.gev_gemm_f64_scratch_bytes.restype = ctypes.c_size_t
    return L, torch, torch.device("cuda:0")


def call(env, M, N, K, ta, tb, alpha, opA, opB, beta, C0, engine):
    L, torch, dev = env
    Astore = opA if ta == 0 else opA.T
    Bstore = opB if tb == 0 else opB.T
    Ab, Bb, Cb = (x.T.contiguous().to(dev) for x in (Astore, Bstore, C0))
    st = torch.zeros(16, dtype=torch.int32, device=dev)
    nbytes = L.gev_gemm_f64_scratch_bytes(M, N, K)
    scr = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    code = L.gev_gemm_f64(M, N, K, ta, tb, alpha, ctypes.c_void_p(Ab.data_ptr()), max(1, Astore.shape[0]),
                          ctypes.c_void_p(Bb.data_ptr()), max(1, Bstore.shape[0]), beta,
                          ctypes.c_void_p(Cb.data_ptr()), max(1, M), engine, ctypes.c_void_p(stream.cuda_stream),
                          ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(scr.data_ptr()), nbytes)
    assert code == 0 and int(st[1].item()) == 0
    return Cb.cpu().T


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
    C = call(env, M, N, K, ta, tb, alpha, opA, opB, beta, C0, engine)
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


def test_gemm_f64_k_above_one_launch(env):
    """K = 40000 runs as two launches (32768 + 7232), the second accumulating onto the first."""
    assert run(env, 40, 24, 40000, 1, 0, 1) <= 4e-15


def test_gemm_f64_zero_k_scales_c(env):
    """K = 0: C = beta C exactly, both engines."""
    L, torch, dev = env
    C0 = torch.randn(33, 17, dtype=torch.float64)
    for engine in (0, 1):
        C = call(env, 33, 17, 0, 0, 0, 2.0, torch.zeros(33, 0, dtype=torch.float64),
                 torch.zeros(0, 17, dtype=torch.float64), -0.5, C0, engine)
        assert torch.equal(C, -0.5 * C0)


def test_gemm_f64_zero_rows_and_exact_integers(env):
    """A zero row / column gives exact zeros; small integer operands give the exact product."""
    L, torch, dev = env
    g = torch.Generator().manual_seed(5)
    opA = torch.randint(-1000, 1000, (150, 700), generator=g).double()
    opB = torch.randint(-1000, 1000, (700, 90), generator=g).double()
    opA[7] = 0.0
    opB[:, 3] = 0.0
    C = call(env, 150, 90, 700, 0, 0, 1.0, opA, opB, 0.0, torch.zeros(150, 90, dtype=torch.float64), 1)
    assert torch.equal(C, opA @ opB)
    assert torch.all(C[7] == 0) and torch.all(C[:, 3] == 0)


def test_gemm_f64_non_finite_entries_give_nan(env):
    """An Inf in row i of op(A) or a NaN in column j of op(B) makes that row / column NaN (engine 1),
    the other outputs stay finite and within the bound."""
    L, torch, dev = env
    g = torch.Generator().manual_seed(9)
    opA = torch.randn(70, 300, generator=g, dtype=torch.float64)
    opB = torch.randn(300, 50, generator=g, dtype=torch.float64)
    opA[5, 17] = float("inf")
    opB[40, 9] = float("nan")
    C = call(env, 70, 50, 300, 0, 1, 1.0, opA, opB, 0.0, torch.zeros(70, 50, dtype=torch.float64), 1)
    assert torch.all(torch.isnan(C[5])) and torch.all(torch.isnan(C[:, 9]))
    mask = torch.ones_like(C, dtype=torch.bool)
    mask[5] = False
    mask[:, 9] = False
    A2, B2 = opA.clone(), opB.clone()
    A2[5] = 0.0
    B2[:, 9] = 0.0
    ref = A2 @ B2
    scale = A2.abs() @ B2.abs()
    assert torch.all(torch.isfinite(C[mask]))
    assert ((C - ref).abs()[mask] / scale[mask]).max().item() <= 4e-15
