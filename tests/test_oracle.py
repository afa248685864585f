"""Pins for the FP64 CPU oracle (runs without a GPU).

Each check ties the oracle to something other than itself: closed forms (the Toeplitz tridiagonal,
diagonal and constructed spectra), invariants (Sturm counts, trace, Frobenius norm, residual and
orthogonality bounds), brute force at n <= 8 (cyclic Jacobi, a third algorithm) and library
cross-checks (numpy / scipy).  Tolerances follow the bounds stated for the method:
|d lambda| <= 1e-11 ||H||_1, residual <= 1e-13 sqrt(n), orthogonality <= 1e-12 sqrt(n).
"""
import numpy as np
import pytest

import oracle
from paper_2502_02460_gb300 import inputs
from tests.pins import herm_from_lower, jacobi_eig, norm1, real_embedding, sturm_count

EPS = np.finfo(np.float64).eps


# ----------------------------------------------------------------------------------------- QL --
@pytest.mark.parametrize("n", [1, 2, 3, 8, 64, 257])
def test_ql_toeplitz_closed_form(n):
    d, e = inputs.tridiag_toeplitz(n)
    w, Z, st = oracle.steql(d, e)
    assert st == 0
    j = np.arange(1, n + 1)
    exact = np.sort(2.0 - 2.0 * np.cos(j * np.pi / (n + 1)))
    assert np.max(np.abs(w - exact)) <= 8 * n * EPS * 4
    # eigenvectors: sin(i j pi/(n+1)), normalised; compare up to sign
    i = np.arange(1, n + 1)
    for col in range(n):
        jj = col + 1  # ascending eigenvalue 2-2cos(j pi/(n+1)) is increasing in j
        v = np.sin(i * jj * np.pi / (n + 1))
        v /= np.linalg.norm(v)
        assert abs(abs(v @ Z[:, col]) - 1.0) < 1e-12


def test_ql_diagonal_returns_sorted_diagonal():
    rng = np.random.default_rng(5)
    d = rng.standard_normal(50)
    w, Z, st = oracle.steql(d, np.zeros(49))
    assert st == 0
    assert np.array_equal(w, np.sort(d))
    assert np.allclose(np.abs(Z), np.eye(50)[:, np.argsort(d, kind="stable")])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ql_sturm_counts(seed):
    d, e = inputs.random_tridiag(120, seed)
    w, Z, st = oracle.steql(d, e)
    assert st == 0
    rng = np.random.default_rng(100 + seed)
    xs = np.concatenate([rng.uniform(w.min() - 1, w.max() + 1, 40), (w[:-1] + w[1:]) / 2])
    for x in xs:
        assert sturm_count(d, e, x) == int(np.sum(w < x))


@pytest.mark.parametrize("n", [2, 5, 8])
def test_ql_jacobi_bruteforce(n):
    d, e = inputs.random_tridiag(n, 40 + n)
    w, Z, st = oracle.steql(d, e)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    wj, Vj = jacobi_eig(T)
    assert np.max(np.abs(w - wj)) <= 1e-13 * max(1, np.abs(wj).max())
    for c in range(n):
        assert abs(abs(Vj[:, c] @ Z[:, c]) - 1) < 1e-10


def test_ql_trace_and_orthogonality():
    d, e = inputs.glued_wilkinson(21, 4, 1e-10)
    w, Z, st = oracle.steql(d, e)
    assert st == 0
    n = len(d)
    assert abs(w.sum() - d.sum()) <= 1e-12 * np.abs(d).sum()
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) <= 1e-13 * n
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    assert np.max(np.abs(T @ Z - Z * w[None, :])) <= 1e-13 * n * norm1(T)


# ----------------------------------------------------------------------------------- Cholesky --
@pytest.mark.parametrize("cx", [False, True])
def test_potrf_diagonal(cx):
    s = np.array([4.0, 9.0, 0.25, 2.0])
    S = np.diag(s).astype(np.complex128 if cx else np.float64)
    L, info = oracle.potrf(S)
    assert info == 0
    assert np.allclose(L, np.diag(np.sqrt(s)), rtol=0, atol=1e-15)


@pytest.mark.parametrize("cx", [False, True])
def test_potrf_recovers_factor(cx):
    rng = np.random.default_rng(3)
    n = 40
    L0 = 0.2 * np.tril(rng.standard_normal((n, n)))
    if cx:
        L0 = L0 + 0.2j * np.tril(rng.standard_normal((n, n)), -1)
    L0[np.diag_indices(n)] = np.abs(L0[np.diag_indices(n)]) + 1.0
    S = L0 @ L0.conj().T
    L, info = oracle.potrf(inputs.lower_only(S))
    assert info == 0
    assert np.max(np.abs(L - L0)) <= 1e-12 * np.abs(L0).max()
    assert np.max(np.abs(L @ L.conj().T - S)) <= 4 * n * EPS * norm1(S)
    assert np.allclose(L, np.linalg.cholesky(S), atol=1e-12)


def test_potrf_not_spd_pivot_index():
    S = np.eye(6)
    S[3, 3] = -1.0
    _, info = oracle.potrf(S)
    assert info == 4
    S = np.eye(5)
    S[2, 1] = S[1, 2] = 1.0  # rows 1 and 2 identical -> zero pivot at index 2
    _, info = oracle.potrf(S)
    assert info == 3


# ---------------------------------------------------------------------------------- reduction --
@pytest.mark.parametrize("cx", [False, True])
def test_reduce_recovers_M(cx):
    rng = np.random.default_rng(11)
    n = 48
    L0 = np.tril(rng.standard_normal((n, n)) * 0.3)
    if cx:
        L0 = L0 + 0.3j * np.tril(rng.standard_normal((n, n)), -1)
    L0[np.diag_indices(n)] = 1.0 + rng.uniform(0, 1, n)
    M = rng.standard_normal((n, n))
    if cx:
        M = M + 1j * rng.standard_normal((n, n))
    M = 0.5 * (M + M.conj().T)
    H = L0 @ M @ L0.conj().T
    S = L0 @ L0.conj().T
    L, info = oracle.potrf(inputs.lower_only(S))
    A, asym = oracle.reduce(inputs.lower_only(H), L)
    assert info == 0
    assert np.max(np.abs(A - M)) <= 1e-11 * np.abs(M).max()
    assert np.allclose(A, A.conj().T, atol=0)


# ---------------------------------------------------------------------------- tridiagonalise --
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 96])
def test_sytrd_invariants(cx, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    if cx:
        A = A + 1j * rng.standard_normal((n, n))
    A = 0.5 * (A + A.conj().T)
    d, e, V, tau = oracle.sytrd(A)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    assert abs(np.trace(A).real - d.sum()) <= 1e-12 * max(1, np.abs(A).sum())
    assert abs(np.linalg.norm(A) - np.linalg.norm(T)) <= 1e-12 * np.linalg.norm(A)
    # eigenvalues: QL on (d, e) vs numpy eigh on A (library cross-check)
    w, Z, st = oracle.steql(d, e)
    assert np.max(np.abs(w - np.linalg.eigvalsh(A))) <= 1e-12 * max(1, norm1(A))
    # Q is unitary and A = Q T Q^H
    Q = oracle.ormtr(V, tau, np.eye(n, dtype=A.dtype))
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(n))) <= 1e-13 * max(n, 1)
    assert np.max(np.abs(Q @ T @ Q.conj().T - A)) <= 1e-12 * max(1, norm1(A))


def test_sytrd_tridiagonal_input_unchanged_up_to_signs():
    d0, e0 = inputs.random_tridiag(30, 9)
    A = np.diag(d0) + np.diag(e0, 1) + np.diag(e0, -1)
    d, e, _, _ = oracle.sytrd(A)
    assert np.allclose(d, d0, atol=1e-15)
    assert np.allclose(np.abs(e), np.abs(e0), atol=1e-15)


def test_sytrd_sturm_counts_match_constructed_spectrum():
    rng = np.random.default_rng(21)
    n = 80
    lam = np.sort(inputs.draw_spectrum(n, rng))
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    d, e, _, _ = oracle.sytrd(A)
    for x in np.concatenate([(lam[:-1] + lam[1:]) / 2, [lam[0] - 1, lam[-1] + 1]]):
        assert sturm_count(d, e, x) == int(np.sum(lam < x))


# ------------------------------------------------------------------------------ whole pencil --
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,k", [(1, 1), (2, 1), (16, 16), (64, 20), (200, 60)])
def test_gev_constructed_spectrum(cx, n, k):
    p = inputs.make_problem(n, k, seed=n, complex_=cx)
    H = inputs.lower_only(p.H)
    S = inputs.lower_only(p.S)
    w, C, info, dg = oracle.gev(H, S, k)
    assert info == 0
    h1 = norm1(p.H)
    assert np.max(np.abs(w - p.lam[:k])) <= 1e-11 * h1
    assert dg["resid"] <= 1e-13 * np.sqrt(n)
    assert dg["ortho"] <= 1e-12 * np.sqrt(n)
    # independent recomputation of the two diagnostics with numpy
    Hf, Sf = p.H, p.S
    R = Hf @ C - Sf @ C * w[None, :]
    assert norm1(R) / (h1 * norm1(C)) <= 1e-13 * np.sqrt(n)
    assert norm1(C.conj().T @ Sf @ C - np.eye(k)) <= 1e-12 * np.sqrt(n)


@pytest.mark.parametrize("cx", [False, True])
def test_gev_config0_recipe_n512(cx):
    n = 512
    p = inputs.make_problem(n, n, seed=0, complex_=cx)
    w, C, info, dg = oracle.gev(p.H, p.S, n)
    assert info == 0
    assert np.max(np.abs(w - p.lam)) <= 1e-11 * norm1(p.H)
    assert dg["resid"] <= 1e-13 * np.sqrt(n)
    assert dg["ortho"] <= 1e-12 * np.sqrt(n)


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n", [1, 3, 6])
def test_gev_bruteforce_small(cx, n):
    """n <= 8: cyclic Jacobi on the real embedding of S^{-1/2} H S^{-1/2}, where S^{-1/2} also comes
    from Jacobi, plus scipy's generalized eigh as a library cross-check."""
    rng = np.random.default_rng(70 + n)
    B = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cx else 0)
    S = B @ B.conj().T + n * np.eye(n)
    G = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cx else 0)
    H = 0.5 * (G + G.conj().T)
    w, C, info, dg = oracle.gev(H, S, n)
    assert info == 0
    Sr, Hr = real_embedding(S), real_embedding(H)
    sig, V = jacobi_eig(Sr)
    Sih = (V / np.sqrt(sig)[None, :]) @ V.T
    wj, _ = jacobi_eig(Sih @ Hr @ Sih)
    if cx:
        wj = wj[::2]
    assert np.max(np.abs(w - wj)) <= 1e-12 * max(1, norm1(H))
    import scipy.linalg

    ws = scipy.linalg.eigh(H, S, eigvals_only=True)
    assert np.max(np.abs(w - ws)) <= 1e-12 * max(1, norm1(H))


def test_gev_scipy_subset_crosscheck():
    import scipy.linalg

    p = inputs.make_problem(300, 90, seed=7, complex_=True)
    w, C, info, dg = oracle.gev(p.H, p.S, 90)
    ws, Cs = scipy.linalg.eigh(p.H, p.S, subset_by_index=[0, 89])
    assert np.max(np.abs(w - ws)) <= 1e-11 * norm1(p.H)
    # same eigenvectors up to phase: |c_i^H S c_s_i| = 1
    ov = np.abs(np.sum(C.conj() * (p.S @ Cs), axis=0))
    assert np.max(np.abs(ov - 1)) <= 1e-9


def test_gev_reads_lower_triangle_only():
    p = inputs.make_problem(40, 12, seed=4)
    w1, C1, _, _ = oracle.gev(p.H, p.S, 12)
    w2, C2, _, _ = oracle.gev(inputs.lower_only(p.H, 1e6), inputs.lower_only(p.S, -3.0), 12)
    assert np.array_equal(w1, w2)
    assert np.array_equal(C1, C2)


def test_gev_not_spd_reports_pivot():
    n = 10
    H = np.eye(n)
    S = np.eye(n)
    S[6, 6] = -2.0
    _, _, info, _ = oracle.gev(H, S, 3)
    assert info == 7


def test_gev_phase_normalisation():
    p = inputs.make_problem(50, 50, seed=12, complex_=True)
    _, C, _, _ = oracle.gev(p.H, p.S, 50)
    for c in range(50):
        i = int(np.argmax(np.abs(C[:, c])))
        assert abs(C[i, c].imag) == 0.0 and C[i, c].real > 0


def test_cluster_recipe():
    p = inputs.make_problem(256, 77, seed=1, cluster=True)
    a = 77 // 2
    assert np.allclose(np.diff(p.lam[a:a + 16]), 1e-8 / 15, rtol=1e-3)
    w, C, info, dg = oracle.gev(p.H, p.S, 77)
    assert info == 0
    assert np.max(np.abs(w - p.lam[:77])) <= 1e-11 * norm1(p.H)
    assert dg["resid"] <= 1e-13 * np.sqrt(256)
    assert dg["ortho"] <= 1e-12 * np.sqrt(256)


def test_oracle_thread_count_invariance():
    """Results do not depend on the OpenMP thread count (each element computed by one thread).
    The inputs are built once here, so only the oracle runs under different thread counts."""
    import os
    import subprocess
    import sys
    import tempfile
    import textwrap

    p = inputs.make_problem(120, 40, seed=3, complex_=True)
    code = textwrap.dedent("""
        import sys, numpy as np, oracle
        z = np.load(sys.argv[1])
        w, C, info, dg = oracle.gev(z['H'], z['S'], 40)
        np.save(sys.argv[2], np.concatenate([w, C.real.ravel(), C.imag.ravel()]))
    """)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "in.npz")
        np.savez(src, H=p.H, S=p.S)
        for t in (1, 3):
            f = os.path.join(td, f"o{t}.npy")
            env = dict(os.environ, OMP_NUM_THREADS=str(t), PYTHONPATH=root)
            subprocess.check_call([sys.executable, "-c", code, src, f], env=env, cwd=root)
            outs.append(np.load(f))
    assert np.array_equal(outs[0], outs[1])


# ------------------------------------------------------------------------------------ density --
def _occupied_problem(cx, n=40, k=12, seed=11):
    p = inputs.make_problem(n, k, seed=seed, complex_=cx)
    w, C, info, _ = oracle.gev(p.H, p.S, k)
    assert info == 0
    return p, w, C


@pytest.mark.parametrize("cx", [False, True])
def test_density_electron_count_and_band_energy(cx):
    """The density integrates to the electron count and to the band energy: with
    S_ij = <phi_i|phi_j>, sum_ij P_ij S_ij = sum_l f_l and sum_ij P_ij H_ij = sum_l f_l lambda_l
    (S-orthonormal orbitals, H c_l = lambda_l S c_l).  For complex data a conjugate on the wrong index
    breaks both (S is not real), as does a dropped weight or a transposed operand."""
    p, w, C = _occupied_problem(cx)
    f = np.random.default_rng(5).uniform(0.0, 2.0, w.size)
    P = oracle.density(C, f)
    PE = oracle.density(C, f * w)
    h1 = norm1(p.H)
    assert abs(np.sum(P * p.S) - f.sum()) <= 1e-12 * f.sum()
    assert abs(np.sum(P * p.H) - np.dot(f, w)) <= 1e-12 * h1 * f.sum()
    assert abs(np.sum(PE * p.S) - np.dot(f, w)) <= 1e-12 * h1 * f.sum()
    assert np.max(np.abs(P - P.conj().T)) <= 1e-15 * np.max(np.abs(P))
    if cx:  # the conjugate on the second index instead gives a different number
        assert abs(np.sum(P.conj() * p.S) - f.sum()) > 1e-6


@pytest.mark.parametrize("cx", [False, True])
def test_density_full_occupation_is_inverse_overlap(cx):
    """k = n, f = 1: C C^H = S^{-1} for square S-orthonormal C, so P = conj(S^{-1}) (numpy's inverse
    as the library cross-check)."""
    n = 24
    p = inputs.make_problem(n, n, seed=4, complex_=cx)
    w, C, info, _ = oracle.gev(p.H, p.S, n)
    assert info == 0
    P = oracle.density(C, np.ones(n))
    Si = np.linalg.inv(p.S)
    assert np.max(np.abs(P - Si.conj())) <= 1e-12 * np.max(np.abs(Si))


@pytest.mark.parametrize("cx", [False, True])
def test_density_idempotent_and_energy_weighted_projection(cx):
    """f in {0, 1}: P conj(S) P = P (McWeeny idempotency in the non-orthogonal basis) and
    PE = P conj(H) P (C^H H C = Lambda on the occupied block)."""
    p, w, C = _occupied_problem(cx, n=36, k=14, seed=8)
    f = np.zeros(w.size)
    f[:9] = 1.0
    P = oracle.density(C, f)
    PE = oracle.density(C, f * w)
    scale = np.max(np.abs(P))
    assert np.max(np.abs(P @ p.S.conj() @ P - P)) <= 1e-12 * scale * norm1(p.S)
    assert np.max(np.abs(P @ p.H.conj() @ P - PE)) <= 1e-12 * scale * norm1(p.H)
    # zero occupation: exactly zero
    assert not np.any(oracle.density(C, np.zeros(w.size)))

