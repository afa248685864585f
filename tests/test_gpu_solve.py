"""GPU parity of the two-stage reduction, the divide-and-conquer solve, the back-transforms and the
whole generalized solve (gev_solve) against the FP64 CPU oracle.

Bounds (the method's stated tolerances): |d lambda| <= 1e-11 ||H||_1; residual
||HC - SC Lambda||_1/(||H||_1 ||C||_1) <= 1e-13 sqrt(n); orthogonality ||C^H S C - I||_1 <=
1e-12 sqrt(n).  Eigenvectors are compared through their S-inner products with the oracle's
(phase free): for eigenvalues separated by a relative gap, |c_gpu^H S c_oracle| = 1 to 1e-8, and
inside clusters the projector onto the cluster's span must agree."""
import numpy as np
import pytest

import oracle
from paper_2502_02460_gb300 import inputs
from tests.parity import compare_to_oracle
from tests.pins import norm1, sturm_count

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


def tridiag(d, e):
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


# --------------------------------------------------------------------------- divide & conquer --
def tri_cases():
    yield "toeplitz", *inputs.tridiag_toeplitz(300)
    yield "random", *inputs.random_tridiag(257, 3)
    yield "wilkinson", *inputs.glued_wilkinson(21, 12, 1e-9)
    d = np.linspace(-1, 1, 100)
    yield "diagonal", d, np.zeros(99)
    yield "tiny", *inputs.random_tridiag(2, 1)
    yield "leaf", *inputs.random_tridiag(32, 2)
    yield "twoleaf", *inputs.random_tridiag(33, 2)
    rng = np.random.default_rng(9)
    dd = np.repeat(rng.standard_normal(25), 8)  # many equal diagonal entries, weak coupling
    yield "clustered", dd, 1e-6 * rng.standard_normal(199)


@pytest.mark.parametrize("case", list(tri_cases()), ids=lambda c: c[0])
def test_stedc_matches_oracle(dev, case):
    import torch

    name, d, e = case
    n = len(d)
    wo, Zo, st = oracle.steql(d, e)
    assert st == 0
    T = tridiag(d, e)
    tn = max(norm1(T), 1e-300)
    for k in sorted({n, max(1, n // 3), 1}):
        with gv().Solver(n, device=dev) as s:
            w, Zb, defl = s.stedc(torch.from_numpy(d).to(dev), torch.from_numpy(e).to(dev), k)
            w = w.cpu().numpy()
            Z = gv().numpy_from_cm(Zb)
        assert np.max(np.abs(w - wo)) <= 1e-13 * tn * np.sqrt(n), name
        R = T @ Z - Z * w[None, :k]
        assert norm1(R) / tn <= 1e-13 * n, name
        assert norm1(Z.T @ Z - np.eye(k)) <= 1e-12 * n, name


@pytest.mark.parametrize("n", [100, 1000])
def test_stedc_sturm(dev, n):
    import torch

    d, e = inputs.random_tridiag(n, 77)
    with gv().Solver(n, device=dev) as s:
        w, _, _ = s.stedc(torch.from_numpy(d).to(dev), torch.from_numpy(e).to(dev), 1)
        w = w.cpu().numpy()
    for x in (w[:-1] + w[1:])[:: max(1, n // 50)] / 2:
        assert sturm_count(d, e, x) == int(np.sum(w < x))


# ------------------------------------------------------------------- two-stage reduction --
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,b", [(3, 16), (40, 16), (130, 32), (300, 64), (517, 32)])
def test_band_and_tridiag_preserve_spectrum(dev, cx, n, b):
    rng = np.random.default_rng(n + b)
    A = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cx else 0)
    A = 0.5 * (A + A.conj().T)
    lam = np.linalg.eigvalsh(A)
    with gv().Solver(n, complex_=cx, device=dev, band_b=b) as s:
        Ab = gv().cm_from_numpy(A, dev)
        used = s.he2hb(Ab, b)
        B = gv().numpy_from_cm(Ab)
        d, e = s.hb2st()
        d = d.cpu().numpy()
        e = e.cpu().numpy()
    assert used == b
    # band structure and spectrum of the band matrix
    Bl = np.tril(B)
    assert np.max(np.abs(np.tril(Bl, -b - 1))) == 0.0
    Bf = Bl + np.tril(Bl, -1).conj().T
    scale = norm1(A)
    assert np.max(np.abs(np.linalg.eigvalsh(Bf) - lam)) <= 1e-13 * n * scale
    # tridiagonal: same spectrum (oracle QL on (d, e)), same trace
    wt, _, st = oracle.steql(d, e)
    assert st == 0
    assert np.max(np.abs(wt - lam)) <= 1e-13 * n * scale
    assert abs(d.sum() - np.trace(A).real) <= 1e-12 * n * scale


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,k,b", [(64, 64, 16), (200, 70, 32), (450, 150, 64), (333, 1, 32)])
def test_standard_problem_chain(dev, cx, n, k, b):
    """he2hb -> hb2st -> stedc -> back on a standard Hermitian A: A Y = Y Lambda, Y^H Y = I."""
    rng = np.random.default_rng(n * 7 + k)
    A = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cx else 0)
    A = 0.5 * (A + A.conj().T)
    with gv().Solver(n, complex_=cx, device=dev, band_b=b) as s:
        s.he2hb(gv().cm_from_numpy(A, dev), b)
        d, e = s.hb2st()
        w, Zb, _ = s.stedc(d, e, k)
        Y = gv().numpy_from_cm(s.back(Zb, k))
        w = w.cpu().numpy()[:k]
    scale = norm1(A)
    assert np.max(np.abs(w - np.linalg.eigvalsh(A)[:k])) <= 1e-13 * n * scale
    assert norm1(A @ Y - Y * w[None, :]) / scale <= 1e-13 * n
    assert norm1(Y.conj().T @ Y - np.eye(k)) <= 1e-12 * n


# ------------------------------------------------------------------------------- whole solve --
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,k", [(1, 1), (2, 2), (3, 1), (64, 64), (100, 33), (200, 200), (333, 100)])
def test_solve_matches_oracle(dev, cx, n, k):
    p = inputs.make_problem(n, k, seed=1000 + n, complex_=cx)
    with gv().Solver(n, complex_=cx, device=dev) as s:
        Hb = gv().cm_from_numpy(inputs.lower_only(p.H, 3.0), dev)
        Sb = gv().cm_from_numpy(inputs.lower_only(p.S, -1.0), dev)
        w, Cb = s.solve_cm(Hb, Sb, k)
        w = w.cpu().numpy()
        C = gv().numpy_from_cm(Cb)
    compare_to_oracle(p, w, C, k)
    # phase convention: the largest-modulus entry of each column is real and positive
    for c in range(k):
        i = int(np.argmax(np.abs(C[:, c])))
        assert C[i, c].real > 0 and abs(C[i, c].imag) <= 1e-300


def test_solve_config0_recipe(dev):
    """The N=512 all-pairs real configuration (seed 0), element-wise against the oracle."""
    n = 512
    p = inputs.make_problem(n, n, seed=0)
    with gv().Solver(n, device=dev) as s:
        w, Cb = s.solve_cm(gv().cm_from_numpy(p.H, dev), gv().cm_from_numpy(p.S, dev), n)
        w = w.cpu().numpy()
        C = gv().numpy_from_cm(Cb)
    compare_to_oracle(p, w, C, n)


@pytest.mark.parametrize("b", [16, 32, 64])
def test_solve_band_widths_and_cluster(dev, b):
    n, k = 700, 210
    p = inputs.make_problem(n, k, seed=1, cluster=True)
    with gv().Solver(n, device=dev, band_b=b) as s:
        w, Cb = s.solve_cm(gv().cm_from_numpy(p.H, dev), gv().cm_from_numpy(p.S, dev), k)
        w = w.cpu().numpy()
        C = gv().numpy_from_cm(Cb)
        rep = s.last_report
    compare_to_oracle(p, w, C, k)
    assert rep["deflated"] >= 0


def test_reuse_factor_matches_fresh_solve(dev):
    n, k = 300, 90
    p = inputs.make_problem(n, k, seed=21, complex_=True)
    rng = np.random.default_rng(5)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    dH = 0.5 * (G + G.conj().T)
    H2 = p.H + 1e-3 * np.linalg.norm(p.H) / np.linalg.norm(dH) * dH
    with gv().Solver(n, complex_=True, device=dev) as s:
        s.reuse_factor(True)
        s.solve_cm(gv().cm_from_numpy(p.H, dev), gv().cm_from_numpy(p.S, dev), k)
        w2, C2 = s.solve_cm(gv().cm_from_numpy(H2, dev), None, k)
        assert s.last_report["reused_factor"] == 1
        w2 = w2.cpu().numpy()
    with gv().Solver(n, complex_=True, device=dev) as s:
        w3, _ = s.solve_cm(gv().cm_from_numpy(H2, dev), gv().cm_from_numpy(p.S, dev), k)
        w3 = w3.cpu().numpy()
    assert np.max(np.abs(w2 - w3)) <= 1e-12 * norm1(H2)
    wo, _, _, _ = oracle.gev(H2, p.S, k)
    assert np.max(np.abs(w2 - wo)) <= 1e-11 * norm1(H2)


def test_reuse_without_factor_is_an_error(dev):
    n = 50
    p = inputs.make_problem(n, 5, seed=2)
    with gv().Solver(n, device=dev) as s:
        s.reuse_factor(True)
        with pytest.raises(gv().GevError) as ei:
            s.solve_cm(gv().cm_from_numpy(p.H, dev), None, 5)
        assert ei.value.code == 6


def test_not_spd_overlap_reports_pivot(dev):
    n = 150
    S = np.eye(n)
    S[97, 97] = -0.5
    H = np.eye(n)
    with gv().Solver(n, device=dev) as s:
        with pytest.raises(gv().GevError) as ei:
            s.solve_cm(gv().cm_from_numpy(H, dev), gv().cm_from_numpy(S, dev), 3)
        assert ei.value.code == 1 and ei.value.info == 98
        # the handle stays usable
        p = inputs.make_problem(n, 10, seed=3)
        w, _ = s.solve_cm(gv().cm_from_numpy(p.H, dev), gv().cm_from_numpy(p.S, dev), 10)
        assert np.max(np.abs(w.cpu().numpy() - p.lam[:10])) <= 1e-11 * norm1(p.H)


@pytest.mark.parametrize("cx", [False, True])
def test_repeated_solves_are_bitwise_identical(dev, cx):
    """A handle keeps no state that changes results: repeated solves, and a fresh handle, agree
    bit for bit (the divide and conquer relies on zero rows outside each eigenvector block)."""
    n, k = 700, 200
    p = inputs.make_problem(n, k, seed=31, complex_=cx)
    Hb, Sb = gv().cm_from_numpy(p.H, dev), gv().cm_from_numpy(p.S, dev)
    outs = []
    with gv().Solver(n, complex_=cx, device=dev) as s:
        for _ in range(3):
            w, Cb = s.solve_cm(Hb, Sb, k)
            outs.append((w.cpu().numpy(), gv().numpy_from_cm(Cb)))
    with gv().Solver(n, complex_=cx, device=dev) as s:
        w, Cb = s.solve_cm(Hb, Sb, k)
        outs.append((w.cpu().numpy(), gv().numpy_from_cm(Cb)))
    for w, C in outs[1:]:
        assert np.array_equal(w, outs[0][0])
        assert np.array_equal(C, outs[0][1])
    assert np.max(np.abs(outs[0][0] - p.lam[:k])) <= 1e-11 * norm1(p.H)


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,k,b", [(100, 33, 16), (333, 100, 32), (700, 210, 64), (1100, 300, 64)])
def test_solve_with_native_fp64_products_matches_oracle(dev, cx, n, k, b):
    """The FP64 solve with every matrix product on the native FP64 tensor path (DMMA,
    fp64_emulation=0; the other solve tests run the default, products emulated on the BF16 tensor
    cores): same bounds.  Covers the triangular operand masks (inversion, Multiply step), conjugate
    transposes, lower-only outputs and split K of both engines."""
    p = inputs.make_problem(n, k, seed=3000 + n, complex_=cx, cluster=(n == 700))
    with gv().Solver(n, complex_=cx, device=dev, band_b=b, fp64_emulation=0) as s:
        w, Cb = s.solve_cm(gv().cm_from_numpy(p.H, dev), gv().cm_from_numpy(p.S, dev), k)
        w = w.cpu().numpy()
        C = gv().numpy_from_cm(Cb)
    compare_to_oracle(p, w, C, k)


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,k,b", [(37, 5, 16), (200, 70, 32), (450, 450, 64), (517, 129, 32), (777, 1, 64)])
def test_back_transform_engines_agree(dev, cx, n, k, b):
    """Back-transform 2 in compact-WY form on the tensor cores (two block-diagonal products per level,
    the default engine) and the reflector-by-reflector level kernel on the FP64 CUDA cores
    (fp64_emulation=0): each gives A Y = Y Lambda and Y^H Y = I to FP64 rounding, and their vectors
    agree (phase free) wherever the eigenvalue is separated from its neighbours."""
    rng = np.random.default_rng(n + 3 * k + b)
    A = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cx else 0)
    A = 0.5 * (A + A.conj().T)
    scale = norm1(A)
    lam = np.linalg.eigvalsh(A)
    Ys = []
    for emu in (1, 0):
        with gv().Solver(n, complex_=cx, device=dev, band_b=b, fp64_emulation=emu) as s:
            s.he2hb(gv().cm_from_numpy(A, dev), b)
            d, e = s.hb2st()
            w, Zb, _ = s.stedc(d, e, k)
            Y = gv().numpy_from_cm(s.back(Zb, k))
            w = w.cpu().numpy()[:k]
        assert norm1(A @ Y - Y * w[None, :]) / scale <= 1e-13 * n
        assert norm1(Y.conj().T @ Y - np.eye(k)) <= 1e-12 * n
        Ys.append(Y)
    G = Ys[0].conj().T @ Ys[1]
    gaps = np.minimum(np.diff(np.concatenate([[-np.inf], lam])), np.diff(np.concatenate([lam, [np.inf]])))[:k]
    for j in range(k):
        if gaps[j] > 1e-3 * scale:
            assert abs(abs(G[j, j]) - 1.0) <= 1e-10
