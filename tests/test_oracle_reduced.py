"""Pins of the oracle's reduced solve for an ill-conditioned overlap (oracle.gev_reduced: the basis
of the eigenvectors of S with eigenvalue >= delta, section "Current Status of the Implementation"),
each against something other than the function itself:

* a constructed pencil with a numerically singular S: S = U diag(sigma) U^H with some sigma below
  delta (down to zero), H = U_m sigma_m^{1/2} Q Lambda Q^H sigma_m^{1/2} U_m^H + U_d G U_d^H (an arbitrary
  Hermitian G on the dropped directions).  The reduced eigenvalues are exactly Lambda, H C = S C Lambda
  holds, C^H S C = I and C has no component along the dropped directions;
* with a well-conditioned S and delta below its smallest eigenvalue nothing is dropped: the result is
  the Cholesky route's (oracle.gev), an independent algorithm for the same pencil;
* brute force at n <= 8: cyclic Jacobi on S, then on the reduced matrix (tests/pins.py);
* the kept count, and k > m reported as an error."""
import numpy as np
import pytest

import oracle
from paper_2502_02460_gb300 import inputs
from tests.pins import jacobi_eig, norm1, real_embedding


def constructed(n, m, cx, seed):
    return inputs.singular_overlap_pencil(n, m, cx, seed)


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,m,k", [(40, 30, 10), (64, 61, 61), (97, 50, 1)])
def test_reduced_constructed_singular_overlap(cx, n, m, k):
    H, S, lam, Ud = constructed(n, m, cx, seed=n + m)
    w, C, mk, st = oracle.gev_reduced(H, S, 1e-5, k)
    assert st == 0 and mk == m
    h1 = norm1(H)
    assert np.max(np.abs(w - lam[:k])) <= 1e-12 * h1
    assert norm1(H @ C - (S @ C) * w[None, :]) <= 1e-12 * h1 * norm1(C)
    assert norm1(C.conj().T @ S @ C - np.eye(k)) <= 1e-12 * n
    assert np.max(np.abs(Ud.conj().T @ C)) <= 1e-9 * np.max(np.abs(C))


@pytest.mark.parametrize("cx", [False, True])
def test_reduced_equals_cholesky_route_when_nothing_is_dropped(cx):
    n, k = 120, 40
    p = inputs.make_problem(n, k, seed=77, complex_=cx)
    w, C, m, st = oracle.gev_reduced(p.H, p.S, 1e-12, k)
    assert st == 0 and m == n
    wo, Co, info, _ = oracle.gev(p.H, p.S, k)
    assert info == 0
    h1 = norm1(p.H)
    assert np.max(np.abs(w - wo)) <= 1e-12 * h1
    assert np.max(np.abs(w - p.lam[:k])) <= 1e-11 * h1
    # both phase normalised: equal vectors (the spectrum is well separated)
    assert np.max(np.abs(C - Co)) <= 1e-9


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,m", [(5, 3), (8, 6)])
def test_reduced_bruteforce_jacobi(cx, n, m):
    H, S, lam, _ = constructed(n, m, cx, seed=7 * n + m)
    k = m
    w, C, mk, st = oracle.gev_reduced(H, S, 1e-5, k)
    assert st == 0 and mk == m
    # Jacobi on the real embedding of S: every eigenvalue twice for complex data
    sj, Vj = jacobi_eig(real_embedding(S))
    step = 2 if cx else 1
    keep = np.nonzero(sj >= 1e-5)[0]
    X = Vj[:, keep] / np.sqrt(sj[keep])[None, :]
    Ht = X.T @ real_embedding(H) @ X
    wj, _ = jacobi_eig(0.5 * (Ht + Ht.T))
    assert np.max(np.abs(w - wj[::step][:k])) <= 1e-11 * norm1(H)


def test_reduced_reports_too_few_kept_vectors():
    H, S, _, _ = constructed(30, 20, False, seed=3)
    w, C, m, st = oracle.gev_reduced(H, S, 1e-5, 25)
    assert st == -3 and m == 20
