"""GPU parity of the individual steps (include/gev_steps.h) against the FP64 CPU oracle.

Sizes span several 64-wide tiles and a ragged tail.  Bounds: the oracle and the GPU are two FP64
routes to the same exact result, so entries agree to a small multiple of n * eps relative to the
norm of the result (well-conditioned Toeplitz overlap, cond(S) ~ 10).  The product-based steps run
with native FP64 products (emu 0) and with products emulated on the BF16 tensor cores (emu 1)."""
import numpy as np
import pytest

import oracle
from paper_2502_02460_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = [1, 7, 64, 65, 200, 333]


@pytest.fixture(scope="module")
def dev():
    import torch

    from paper_2502_02460_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def solver(n, cx, dev, **kw):
    from paper_2502_02460_gb300 import gev

    return gev.Solver(n, complex_=cx, device=dev, **kw)


def to_dev(M, dev):
    from paper_2502_02460_gb300 import gev

    return gev.cm_from_numpy(M, dev)


def to_np(B):
    from paper_2502_02460_gb300 import gev

    return gev.numpy_from_cm(B)


@pytest.mark.parametrize("emu", [0, 1])
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n", SIZES)
def test_potrf_matches_oracle(dev, cx, n, emu):
    p = inputs.make_problem(n, 1, seed=n, complex_=cx)
    S = inputs.lower_only(p.S, 7.0)  # upper triangle must not be read
    Lo, info = oracle.potrf(p.S)
    assert info == 0
    with solver(n, cx, dev, fp64_emulation=emu) as s:
        B = to_dev(S, dev)
        assert s.potrf(B) == 0
        L = to_np(B)
    assert np.max(np.abs(L - Lo)) <= 64 * n * np.finfo(float).eps * np.abs(Lo).max()
    assert np.all(np.triu(L, 1) == 0)


def test_potrf_not_spd_reports_first_pivot(dev):
    for n, bad in ((10, 6), (150, 131), (200, 64)):
        S = np.eye(n)
        S[bad, bad] = -1.0
        S[bad + 1:, bad + 1:] *= -1.0  # later pivots bad too: the first one must be reported
        with solver(n, False, dev) as s:
            B = to_dev(S, dev)
            assert s.potrf(B) == bad + 1


@pytest.mark.parametrize("emu", [0, 1])
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n", SIZES)
def test_trtri_inverts(dev, cx, n, emu):
    p = inputs.make_problem(n, 1, seed=n + 1, complex_=cx)
    Lo, _ = oracle.potrf(p.S)
    with solver(n, cx, dev, fp64_emulation=emu) as s:
        B = to_dev(Lo, dev)
        s.trtri(B)
        X = to_np(B)
    eye = np.eye(n)
    assert np.max(np.abs(X @ Lo - eye)) <= 64 * n * np.finfo(float).eps * max(1, np.abs(X).max())
    assert np.all(np.triu(X, 1) == 0)


@pytest.mark.parametrize("emu", [0, 1])
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n", SIZES)
def test_hegst_matches_oracle(dev, cx, n, emu):
    p = inputs.make_problem(n, 1, seed=n + 2, complex_=cx)
    Lo, _ = oracle.potrf(p.S)
    Ao, _ = oracle.reduce(p.H, Lo)
    X = np.linalg.inv(Lo)
    X = np.tril(X)
    with solver(n, cx, dev, fp64_emulation=emu) as s:
        A = to_np(s.hegst(to_dev(inputs.lower_only(p.H, -5.0), dev), to_dev(X, dev)))
    assert np.max(np.abs(A - Ao)) <= 1e-12 * np.abs(Ao).max() * max(1, np.sqrt(n))
    assert np.array_equal(A, A.conj().T)


@pytest.mark.parametrize("emu", [0, 1])
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,k", [(1, 1), (65, 3), (200, 130), (333, 333)])
def test_mult(dev, cx, n, k, emu):
    rng = np.random.default_rng(n + k)
    X = np.tril(rng.standard_normal((n, n)))
    Y = rng.standard_normal((n, k))
    if cx:
        X = X + 1j * np.tril(rng.standard_normal((n, n)))
        Y = Y + 1j * rng.standard_normal((n, k))
    with solver(n, cx, dev, fp64_emulation=emu) as s:
        C = to_np(s.mult(to_dev(X, dev), to_dev(Y, dev), k))
    ref = X.conj().T @ Y
    assert np.max(np.abs(C - ref)) <= 1e-13 * n * np.abs(ref).max()


def test_full_chain_reduction_n1000(dev):
    """Steps 1-3 chained on the GPU at a size spanning 16 tiles: A = L^{-1} H L^{-H} vs oracle."""
    n = 1000
    p = inputs.make_problem(n, 1, seed=5)
    Lo, _ = oracle.potrf(p.S)
    Ao, _ = oracle.reduce(p.H, Lo)
    with solver(n, False, dev) as s:
        B = to_dev(p.S, dev)
        assert s.potrf(B) == 0
        s.trtri(B)
        A = to_np(s.hegst(to_dev(p.H, dev), B))
    assert np.max(np.abs(A - Ao)) <= 1e-11 * np.abs(Ao).max()
