"""GPU parity of the one-stage Householder tridiagonalisation (the ELPA1 form of the section
"Usability and Tutorials"), its back-transform, and the generalized solve that uses them, against
the FP64 CPU oracle.

The oracle's one-stage reduction (``oracle.sytrd``) takes the same reflector convention (v(0) = 1,
e_j = -sign(Re alpha) ||x||, real), so the GPU's tridiagonal T is the same matrix: d and e are
compared entry by entry, to 1e-12 ||A||_1 (two FP64 routes, well-separated Gaussian spectra), and
the back-transform Y = Q Z against ``oracle.ormtr`` applied to the same Z, entry by entry.  Orders
span several 64-wide symv tiles and panels with ragged tails; panel widths 16, 32 and 64.  Whole
solves: the bounds of ``tests/parity.py`` (|d lambda| <= 1e-11 ||H||_1, residual <= 1e-13 sqrt(n),
S-orthogonality <= 1e-12 sqrt(n), vectors phase-free against the oracle's)."""
import numpy as np
import pytest

import oracle
from paper_2502_02460_gb300 import inputs
from tests.parity import compare_to_oracle
from tests.pins import norm1

pytestmark = pytest.mark.gpu

GEV_ERR_UNSUPPORTED = 7


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


def herm(n, cx, seed):
    rng = np.random.default_rng(seed)
    G = inputs.gaussian(n, rng, cx)
    return (G + G.conj().T) / 2


@pytest.mark.parametrize("b", [16, 32, 64])
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 65, 130, 333])
def test_he2td_matches_oracle(dev, n, cx, b):
    g = gv()
    A = herm(n, cx, 100 + n)
    do, eo, V, tau = oracle.sytrd(A)
    with g.Solver(n, complex_=cx, device=dev, band_b=b, one_stage=True) as s:
        Ab = g.cm_from_numpy(A, dev)
        d, e = s.he2td(Ab)
        d = d.cpu().numpy()
        e = e.cpu().numpy()
    a1 = norm1(A)
    assert np.max(np.abs(d - do)) <= 1e-12 * a1
    if n > 1:
        assert np.max(np.abs(e - eo)) <= 1e-12 * a1
        T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
        assert np.max(np.abs(np.linalg.eigvalsh(T) - np.linalg.eigvalsh(A))) <= 1e-12 * a1


@pytest.mark.parametrize("b", [16, 64])
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,k", [(65, 65), (200, 37), (333, 333)])
def test_one_stage_back_transform_matches_oracle(dev, n, k, cx, b):
    """Y = Q Z for the GPU's own Z: against the oracle's reflectors applied to the same Z."""
    import torch

    g = gv()
    A = herm(n, cx, 7 + n)
    _, _, V, tau = oracle.sytrd(A)
    with g.Solver(n, complex_=cx, device=dev, band_b=b, one_stage=True) as s:
        Ab = g.cm_from_numpy(A, dev)
        d, e = s.he2td(Ab)
        w, Zb, _ = s.stedc(d, e, k)
        Yb = s.back(Zb, k)
        Z = g.numpy_from_cm(Zb)
        Y = g.numpy_from_cm(Yb)
        torch.cuda.synchronize()
    Yo = oracle.ormtr(V, tau, Z.astype(A.dtype))
    assert np.max(np.abs(Y - Yo)) <= 1e-12 * np.sqrt(n)
    wv = w.cpu().numpy()[:k]
    a1 = norm1(A)
    assert np.max(np.abs(A @ Y - Y * wv)) <= 1e-12 * a1
    assert np.max(np.abs(Y.conj().T @ Y - np.eye(k))) <= 1e-12 * np.sqrt(n)


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,k,b", [(7, 7, 64), (130, 130, 32), (333, 83, 64), (512, 512, 64), (700, 175, 16)])
def test_one_stage_solve_matches_oracle(dev, n, k, b, cx):
    g = gv()
    p = inputs.make_problem(n, k, seed=21 + n, complex_=cx)
    with g.Solver(n, complex_=cx, device=dev, band_b=b, one_stage=True, timing=1) as s:
        w, Cb = s.solve_cm(g.cm_from_numpy(inputs.lower_only(p.H, 3.0), dev),
                           g.cm_from_numpy(inputs.lower_only(p.S, -3.0), dev), k)
        rep = s.last_report
        w, C = w.cpu().numpy(), g.numpy_from_cm(Cb)
    compare_to_oracle(p, w, C, k)
    # the one-stage route has no band stage and one back-transform
    assert rep["ms"]["to_band"] == pytest.approx(0.0, abs=0.05)
    assert rep["ms"]["back_band"] == pytest.approx(0.0, abs=0.05)


def test_one_stage_is_deterministic_and_agrees_with_two_stage(dev):
    g = gv()
    n, k = 400, 400
    p = inputs.make_problem(n, k, seed=5, complex_=True)
    H, S = g.cm_from_numpy(p.H, dev), g.cm_from_numpy(p.S, dev)
    with g.Solver(n, complex_=True, device=dev, one_stage=True) as s:
        w1, C1 = s.solve_cm(H, S, k)
        w2, C2 = s.solve_cm(H, S, k)
    assert (w1 == w2).all() and (C1 == C2).all()
    with g.Solver(n, complex_=True, device=dev, one_stage=False) as s:
        w3, _ = s.solve_cm(H, S, k)
    assert float((w1 - w3).abs().max()) <= 1e-11 * norm1(p.H)


def test_one_stage_with_complex_mixed_form_is_unsupported(dev):
    g = gv()
    n = 64
    p = inputs.make_problem(n, 8, seed=1, complex_=True)
    with g.Solver(n, complex_=True, device=dev, mixed=True, one_stage=True) as s:
        with pytest.raises(g.GevError) as ei:
            s.solve_cm(g.cm_from_numpy(p.H, dev), g.cm_from_numpy(p.S, dev), 8)
    assert ei.value.code == GEV_ERR_UNSUPPORTED


@pytest.mark.parametrize("cx", [False, True])
def test_one_stage_reduced_solve_matches_oracle(dev, cx):
    g = gv()
    n, m, k = 160, 150, 40
    H, S, lam, Ud = inputs.singular_overlap_pencil(n, m, cx, seed=4)
    delta = 1e-5
    wo, Co, mo, st = oracle.gev_reduced(H, S, delta, k)
    assert st == 0
    with g.Solver(n, complex_=cx, device=dev, one_stage=True) as s:
        w, _, mk = s.solve_reduced_cm(g.cm_from_numpy(H, dev), g.cm_from_numpy(S, dev), delta, k)
    assert mk == mo
    assert np.max(np.abs(w.cpu().numpy() - wo)) <= 1e-11 * norm1(H)


@pytest.mark.parametrize("n,k,cluster", [(700, 175, False), (1100, 275, True), (1300, 1300, False)])
def test_one_stage_mixed_matches_oracle(dev, n, k, cluster):
    """Real mixed form on the FP32 one-stage reduction: the refinement reaches the same bounds."""
    g = gv()
    p = inputs.make_problem(n, k, seed=31 + n, cluster=cluster)
    with g.Solver(n, device=dev, mixed=True, one_stage=True, timing=1) as s:
        w, Cb = s.solve_cm(g.cm_from_numpy(p.H, dev), g.cm_from_numpy(p.S, dev), k)
        rep = s.last_report
        w, C = w.cpu().numpy(), g.numpy_from_cm(Cb)
    compare_to_oracle(p, w, C, k, resid_bound=1e-11)
    assert rep["refine_resid"] <= 1e-11
    assert rep["ms"]["to_band"] < 0.5 and rep["ms"]["back_band"] < 0.5
