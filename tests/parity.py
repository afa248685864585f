"""Element-wise comparison of a GPU solution of H C = S C Lambda (Eq. 2) with the FP64 CPU oracle.

Bounds (the method's stated tolerances): |d lambda| <= 1e-11 ||H||_1 against the oracle and against
the constructed spectrum; residual ||HC - SC Lambda||_1/(||H||_1 ||C||_1) <= 1e-13 sqrt(n) for the
plain form (1e-11 for the mixed form's refinement target); orthogonality ||C^H S C - I||_1 <=
1e-12 sqrt(n).  Eigenvectors are compared through their S-inner products with the oracle's (phase
free): for an eigenvalue separated from its neighbours by more than 1e-6 ||H||_1,
|c_gpu^H S c_oracle| = 1 to ``tol_vec``; inside a group of closer eigenvalues the singular values of
the group's overlap block must be 1 (the projectors onto the group's span agree)."""
import numpy as np

import oracle
from tests.pins import norm1


def compare_to_oracle(p, w, C, k, tol_vec=1e-8, resid_bound=None, ref=None):
    """p: the inputs.Problem; (w, C): the GPU result; ref: a precomputed oracle.gev(p.H, p.S, k)."""
    wo, Co, info, dg = ref if ref is not None else oracle.gev(p.H, p.S, k)
    assert info == 0
    h1 = norm1(p.H)
    n = p.n
    assert np.max(np.abs(w - wo)) <= 1e-11 * h1
    assert np.max(np.abs(w - p.lam[:k])) <= 1e-11 * h1
    r, o = oracle.check(p.H, p.S, w, C)
    assert r <= (resid_bound if resid_bound is not None else 1e-13 * np.sqrt(n)), r
    assert o <= 1e-12 * np.sqrt(n), o
    G = Co.conj().T @ (p.S @ C)  # k x k overlaps
    groups = []
    start = 0
    for i in range(1, k + 1):
        if i == k or wo[i] - wo[i - 1] > 1e-6 * h1:
            groups.append((start, i))
            start = i
    for a, bnd in groups:
        if bnd - a == 1:
            assert abs(abs(G[a, a]) - 1.0) <= tol_vec, (a, abs(G[a, a]))
        else:
            sv = np.linalg.svd(G[a:bnd, a:bnd], compute_uv=False)
            assert np.max(np.abs(sv - 1.0)) <= 1e-6, (a, bnd)
    return r, o
