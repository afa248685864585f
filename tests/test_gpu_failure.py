"""Failure paths, exercised without a GPU fault: every bounded device wait gives up after its limit
and the call reports an error with the handle still usable; an iteration cap reports
GEV_ERR_NO_CONVERGENCE.

* Timeout: the bulge chasing (band -> tridiagonal, whose sweeps wait on each other's progress flags)
  is asked to wait on a flag that nothing sets (gev_opts.debug_stall) with a short wait limit
  (gev_opts.wait_limit); the kernel must return, the solve must report GEV_ERR_TIMEOUT, and the same
  handle must then solve correctly.
* No convergence: the mixed form's refinement capped at one iteration with an unreachable tolerance.
* The accuracy report of gev_check against the oracle's measurement on a planted wrong answer."""
import numpy as np
import pytest

import oracle
from paper_2502_02460_gb300 import inputs
from tests.pins import norm1

pytestmark = pytest.mark.gpu

GEV_ERR_NO_CONVERGENCE, GEV_ERR_TIMEOUT = 2, 3


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


@pytest.mark.parametrize("cx,mixed", [(False, False), (True, False), (False, True)])
def test_stalled_bulge_chase_times_out_and_handle_recovers(dev, cx, mixed):
    import torch

    n, k = 600, 100
    p = inputs.make_problem(n, k, seed=41, complex_=cx)
    Hb, Sb = gv().cm_from_numpy(p.H, dev), gv().cm_from_numpy(p.S, dev)
    with gv().Solver(n, complex_=cx, device=dev, mixed=mixed, wait_limit=20000, debug_stall=True) as s:
        with pytest.raises(gv().GevError) as ei:
            s.solve_cm(Hb, Sb, k)
        assert ei.value.code == GEV_ERR_TIMEOUT
        torch.cuda.synchronize()  # the context is healthy: no kernel is left running
        # the same handle still works: its Cholesky step against the oracle's
        Ab = gv().cm_from_numpy(p.S, dev)
        assert s.potrf(Ab) == 0
        Lo, info = oracle.potrf(p.S)
        assert info == 0
        Lg = gv().numpy_from_cm(Ab)
        assert np.max(np.abs(Lg - np.tril(Lo))) <= 64 * n * np.finfo(float).eps * np.abs(Lo).max()
    # and a handle without the stall, on the same context, solves correctly
    with gv().Solver(n, complex_=cx, device=dev, mixed=mixed, wait_limit=20000) as s:
        w, _ = s.solve_cm(Hb, Sb, k)
        assert np.max(np.abs(w.cpu().numpy() - p.lam[:k])) <= 1e-11 * norm1(p.H)


def test_refinement_cap_reports_no_convergence(dev):
    n, k = 400, 100
    p = inputs.make_problem(n, k, seed=43)
    Hb, Sb = gv().cm_from_numpy(p.H, dev), gv().cm_from_numpy(p.S, dev)
    with gv().Solver(n, device=dev, mixed=True, refine_max_iter=1, refine_tol=1e-300) as s:
        with pytest.raises(gv().GevError) as ei:
            s.solve_cm(Hb, Sb, k)
        assert ei.value.code == GEV_ERR_NO_CONVERGENCE
        assert s.last_report["refine_iters"] == 2  # iteration 0 and the capped one
    with gv().Solver(n, device=dev, mixed=True) as s:  # the default cap converges
        w, _ = s.solve_cm(Hb, Sb, k)
        assert np.max(np.abs(w.cpu().numpy() - p.lam[:k])) <= 1e-11 * norm1(p.H)


@pytest.mark.parametrize("cx", [False, True])
def test_check_measures_a_planted_wrong_answer(dev, cx):
    """gev_check on eigenpairs with planted errors (one vector perturbed, one eigenvalue shifted)
    reports the residual and orthogonality the oracle measures on the same data."""
    import torch

    n, k = 300, 60
    p = inputs.make_problem(n, k, seed=47, complex_=cx)
    wo, Co, info, _ = oracle.gev(p.H, p.S, k)
    rng = np.random.default_rng(3)
    C = Co.copy()
    C[:, 7] += 1e-6 * rng.standard_normal(n)
    w = wo.copy()
    w[11] += 1e-7
    r_o, o_o = oracle.check(p.H, p.S, w, C)
    with gv().Solver(n, complex_=cx, device=dev) as s:
        r, o = s.check(gv().cm_from_numpy(inputs.lower_only(p.H, 9.0), dev),
                       gv().cm_from_numpy(inputs.lower_only(p.S, -9.0), dev),
                       torch.from_numpy(w).to(dev), gv().cm_from_numpy(C, dev))
    assert r_o > 1e-10 and o_o > 1e-7  # the planted errors dominate
    assert abs(r - r_o) <= 1e-6 * r_o and abs(o - o_o) <= 1e-6 * o_o
