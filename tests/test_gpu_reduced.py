"""GPU parity of the solve for an ill-conditioned overlap (gev_solve_reduced: the pencil in the basis
of the eigenvectors of S with eigenvalue >= delta, section "Current Status of the Implementation")
against the FP64 CPU oracle's reduced solve (oracle.gev_reduced) on the same seeded pencils.

Bounds: |d lambda| <= 1e-11 ||H||_1 against the oracle and the construction; C^H S C = I to
1e-12 sqrt(n); H C = S C Lambda to 1e-12 ||H||_1 ||C||_1; no component of C along the omitted
directions; each vector phase-free against the oracle's for separated eigenvalues; the same kept
count m."""
import numpy as np
import pytest

import oracle
from paper_2502_02460_gb300 import inputs
from tests.pins import norm1

pytestmark = pytest.mark.gpu

GEV_ERR_RANK = 9


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


def compare(H, S, w, C, m, k, lam, Ud, delta):
    """lam / Ud: the construction's exact eigenvalues and omitted directions (None when unknown).
    The residual is checked on the kept space: H C - S C Lambda has no component there (on the
    omitted directions it is whatever H couples into them; zero for the constructed H)."""
    wo, Co, mo, st = oracle.gev_reduced(H, S, delta, k)
    assert st == 0 and m == mo
    h1 = norm1(H)
    n = H.shape[0]
    assert np.max(np.abs(w - wo)) <= 1e-11 * h1
    if lam is not None:
        assert np.max(np.abs(w - lam[:k])) <= 1e-11 * h1
    assert norm1(C.conj().T @ S @ C - np.eye(k)) <= 1e-12 * np.sqrt(n)
    sig, D = np.linalg.eigh(S)
    Dk = D[:, sig >= delta]
    R = H @ C - (S @ C) * w[None, :]
    assert norm1(Dk.conj().T @ R) <= 1e-12 * h1 * norm1(C)
    if lam is not None:
        assert norm1(R) <= 1e-12 * h1 * norm1(C)
    if Ud is not None and Ud.shape[1]:
        assert np.max(np.abs(Ud.conj().T @ C)) <= 1e-9 * np.max(np.abs(C))
    G = Co.conj().T @ (S @ C)
    gaps = np.minimum(np.diff(np.concatenate([[-np.inf], wo])), np.diff(np.concatenate([wo, [np.inf]])))
    for j in range(k):
        if gaps[j] > 1e-6 * h1:
            assert abs(abs(G[j, j]) - 1.0) <= 1e-8


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,m,k", [(40, 30, 10), (200, 150, 150), (517, 400, 97), (64, 63, 1)])
def test_reduced_singular_overlap_matches_oracle(dev, cx, n, m, k):
    H, S, lam, Ud = inputs.singular_overlap_pencil(n, m, cx, seed=n + 7 * m)
    with gv().Solver(n, complex_=cx, device=dev) as s:
        w, Cb, mk = s.solve_reduced_cm(gv().cm_from_numpy(inputs.lower_only(H, 4.0), dev),
                                       gv().cm_from_numpy(inputs.lower_only(S, -4.0), dev), 1e-5, k)
        w, C = w.cpu().numpy(), gv().numpy_from_cm(Cb)
    compare(H, S, w, C, mk, k, lam, Ud, 1e-5)


@pytest.mark.parametrize("cx", [False, True])
def test_reduced_equals_cholesky_route_on_a_well_conditioned_overlap(dev, cx):
    n, k = 300, 90
    p = inputs.make_problem(n, k, seed=61, complex_=cx)
    Hb, Sb = gv().cm_from_numpy(p.H, dev), gv().cm_from_numpy(p.S, dev)
    with gv().Solver(n, complex_=cx, device=dev) as s:
        w, Cb, m = s.solve_reduced_cm(Hb, Sb, 1e-12, k)
        w, C = w.cpu().numpy(), gv().numpy_from_cm(Cb)
        w2, Cb2 = s.solve_cm(Hb, Sb, k)
        w2, C2 = w2.cpu().numpy(), gv().numpy_from_cm(Cb2)
    assert m == n
    compare(p.H, p.S, w, C, m, k, p.lam, None, 1e-12)
    assert np.max(np.abs(w - w2)) <= 1e-11 * norm1(p.H)
    assert np.max(np.abs(C - C2)) <= 1e-8  # both phase normalised, separated spectrum


def test_reduced_reuse_and_rank_errors(dev):
    n, m, k = 150, 100, 40
    H, S, lam, Ud = inputs.singular_overlap_pencil(n, m, False, seed=5)
    rng = np.random.default_rng(1)
    G = rng.standard_normal((n, n))
    H2 = H + 1e-3 * np.linalg.norm(H) / np.linalg.norm(G + G.T) * (G + G.T)
    with gv().Solver(n, device=dev) as s:
        with pytest.raises(gv().GevError) as ei:
            s.solve_reduced_cm(gv().cm_from_numpy(H, dev), None, 1e-5, k)
        assert ei.value.code == 6  # no resident basis yet
        s.reuse_factor(True)
        s.solve_reduced_cm(gv().cm_from_numpy(H, dev), gv().cm_from_numpy(S, dev), 1e-5, k)
        w2, Cb2, m2 = s.solve_reduced_cm(gv().cm_from_numpy(H2, dev), None, 1e-5, k)
        assert s.last_report["reused_factor"] == 1 and m2 == m
        w2, C2 = w2.cpu().numpy(), gv().numpy_from_cm(Cb2)
        # the Cholesky route's resident factor is a different one
        with pytest.raises(gv().GevError) as ei:
            s.solve_cm(gv().cm_from_numpy(H2, dev), None, k)
        assert ei.value.code == 6
        with pytest.raises(gv().GevError) as ei:
            s.solve_reduced_cm(gv().cm_from_numpy(H, dev), gv().cm_from_numpy(S, dev), 1e-5, m + 1)
        assert ei.value.code == GEV_ERR_RANK and ei.value.info == m
    compare(H2, S, w2, C2, m2, k, None, Ud, 1e-5)
