"""GPU parity of the density-matrix output (gev_density): P_ij = sum_l f_l conj(C_il) C_jl and the
energy-weighted PE (weights f_l lambda_l), section "Circumventing the eigenvalue problem" and section
"ELSI", against the oracle's plain definition.

Element bound: the products run on the FP64 matrix-product engine (exact BF16 digit planes with an
error below about 2^-49 of the row / column scales, or native FP64), so
|P_ij - P'_ij| <= 1e-14 k max_l |g_l C_il| max_l |C_jl| (a factor of ten above the engine's bound).
The two triangles are written from the same value: P must be exactly Hermitian."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2502_02460_gb300 import inputs
from tests.pins import norm1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch

    from paper_2502_02460_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def gv():
    from paper_2502_02460_gb300 import gev

    return gev


def bound(C, g):
    k = C.shape[1]
    rw = np.max(np.abs(C) * np.abs(g)[None, :], axis=1)
    rc = np.max(np.abs(C), axis=1)
    return 1e-14 * k * rw[:, None] * rc[None, :]


def random_orbitals(n, k, cx, seed):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((n, k)) + (1j * rng.standard_normal((n, k)) if cx else 0)
    return C, rng.uniform(0.0, 2.0, k), rng.standard_normal(k)


@pytest.mark.parametrize("emu", [1, 0])
@pytest.mark.parametrize("cx,n,k", [(False, 300, 77), (True, 200, 50), (False, 257, 257), (True, 130, 1),
                                    (False, 1, 1), (True, 129, 129), (False, 520, 33)])
def test_density_matches_definition(dev, cx, n, k, emu):
    import torch

    gev = gv()
    C, f, lam = random_orbitals(n, k, cx, seed=n + k)
    with gev.Solver(n, complex_=cx, device=dev, fp64_emulation=emu) as s:
        Cb = gev.cm_from_numpy(C.astype(np.complex128 if cx else np.float64), dev)
        P, PE = s.density(Cb, torch.from_numpy(f), torch.from_numpy(lam))
        torch.cuda.synchronize()
        P, PE = gev.numpy_from_cm(P), gev.numpy_from_cm(PE)
    for got, g in ((P, f), (PE, f * lam)):
        want = oracle.density(C, g)
        err = np.abs(got - want)
        assert np.all(err <= bound(C, g)), float(np.max(err / np.maximum(bound(C, g), 1e-300)))
        assert np.array_equal(got, got.conj().T)  # both triangles from one value, real diagonal


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("cx", [False, True])
def test_density_of_solved_orbitals(dev, cx, mixed):
    """Orbitals from gev_solve: the electron count sum_ij P_ij S_ij = sum_l f_l and the band energy
    sum_ij P_ij H_ij = sum_l f_l lambda_l hold, and P agrees with the oracle's P of the oracle's own
    eigenvectors (P does not depend on the phase of each orbital)."""
    import torch

    gev = gv()
    n, k = 256, 60
    p = inputs.make_problem(n, k, seed=21, complex_=cx)
    f = np.where(np.arange(k) < 40, 2.0, 0.25)
    with gev.Solver(n, complex_=cx, device=dev, mixed=mixed) as s:
        w, Cb = s.solve_cm(gev.cm_from_numpy(p.H, dev), gev.cm_from_numpy(p.S, dev), k)
        P, PE = s.density(Cb, torch.from_numpy(f), w)
        torch.cuda.synchronize()
        w = w.cpu().numpy()
        C = gev.numpy_from_cm(Cb)
        P, PE = gev.numpy_from_cm(P), gev.numpy_from_cm(PE)
    h1 = norm1(p.H)
    assert abs(np.sum(P * p.S) - f.sum()) <= 1e-10 * f.sum()
    assert abs(np.sum(P * p.H) - np.dot(f, w)) <= 1e-10 * h1 * f.sum()
    assert abs(np.sum(PE * p.S) - np.dot(f, w)) <= 1e-10 * h1 * f.sum()
    wo, Co, info, _ = oracle.gev(p.H, p.S, k)
    assert info == 0
    Po = oracle.density(Co, f)
    # an orbital off by a residual r mixes with its neighbours by about r ||H|| / gap; P changes only
    # through mixing across a change of f (after index 40 and at k)
    r, _ = oracle.check(p.H, p.S, w, C)
    gap = min(p.lam[40] - p.lam[39], p.lam[k] - p.lam[k - 1]) / h1
    assert np.max(np.abs(P - Po)) <= (1e-12 + 50.0 * r / gap) * np.max(np.abs(Po))


def test_density_edge_cases(dev):
    import torch

    gev = gv()
    n, k = 70, 20
    C, f, lam = random_orbitals(n, k, True, seed=3)
    with gev.Solver(n, complex_=True, device=dev) as s:
        Cb = gev.cm_from_numpy(C, dev)
        # zero occupation: exactly zero; the NaN prefill of both triangles is overwritten
        P0 = torch.full((n, n), float("nan"), dtype=torch.complex128, device=dev)
        s.density(Cb, torch.zeros(k, dtype=torch.float64), P=P0)
        torch.cuda.synchronize()
        assert torch.all(P0 == 0).item()
        # no energy-weighted matrix requested: only P, the same values as with PE
        P1 = s.density(Cb, torch.from_numpy(f))
        P2, _ = s.density(Cb, torch.from_numpy(f), torch.from_numpy(lam))
        torch.cuda.synchronize()
        assert torch.equal(P1, P2)


def test_density_argument_errors(dev):
    import torch

    gev = gv()
    L = gev.lib()
    n, k = 40, 5
    with gev.Solver(n, device=dev) as s:
        C = torch.zeros((k, n), dtype=torch.float64, device=dev)
        occ = torch.ones(k, dtype=torch.float64, device=dev)
        P = torch.empty((n, n), dtype=torch.float64, device=dev)
        PE = torch.empty((n, n), dtype=torch.float64, device=dev)
        vp = ctypes.c_void_p
        c, o, p, pe = (vp(t.data_ptr()) for t in (C, occ, P, PE))
        nul = vp(0)
        assert L.gev_density(nul, k, c, n, o, o, p, n, pe, n) == -1
        assert L.gev_density(s.h, 0, c, n, o, o, p, n, pe, n) == -2
        assert L.gev_density(s.h, n + 1, c, n, o, o, p, n, pe, n) == -2
        assert L.gev_density(s.h, k, nul, n, o, o, p, n, pe, n) == -3
        assert L.gev_density(s.h, k, c, n - 1, o, o, p, n, pe, n) == -4
        assert L.gev_density(s.h, k, c, n, nul, o, p, n, pe, n) == -5
        assert L.gev_density(s.h, k, c, n, o, nul, p, n, pe, n) == -6
        assert L.gev_density(s.h, k, c, n, o, o, nul, n, pe, n) == -7
        assert L.gev_density(s.h, k, c, n, o, o, p, n - 1, pe, n) == -8
        assert L.gev_density(s.h, k, c, n, o, o, p, n, p, n) == -9
        assert L.gev_density(s.h, k, c, n, o, o, p, n, pe, n - 1) == -10
        assert L.gev_density(s.h, k, c, n, o, nul, p, n, nul, 0) == 0


def test_density_keeps_the_resident_factor(dev):
    """gev_density uses scratch only: a solve that reuses the resident L^{-1} afterwards gives the
    result of the solve before it."""
    import torch

    gev = gv()
    n, k = 192, 40
    p = inputs.make_problem(n, k, seed=5)
    Hb, Sb = gev.cm_from_numpy(p.H, dev), gev.cm_from_numpy(p.S, dev)
    with gev.Solver(n, device=dev) as s:
        s.reuse_factor(True)
        w1, C1 = s.solve_cm(Hb, Sb, k)
        w1, C1 = w1.clone(), C1.clone()
        s.density(C1, torch.ones(k, dtype=torch.float64), w1)
        w2, C2 = s.solve_cm(Hb, None, k)
        torch.cuda.synchronize()
        assert s.last_report["reused_factor"] == 1
        assert torch.max(torch.abs(w2 - w1)).item() <= 1e-12 * norm1(p.H)
        assert torch.max(torch.abs(C2 - C1)).item() <= 1e-10
