"""Independent reference routines used to pin the oracle (no code shared with the oracle or the
GPU path): Sturm counts, cyclic Jacobi, real embedding of Hermitian matrices."""
import numpy as np


def sturm_count(d, e, x):
    """Number of eigenvalues of the symmetric tridiagonal (d, e) strictly below x
    (signs of the LDL^T pivots of T - x I)."""
    n = len(d)
    cnt = 0
    q = 1.0
    tiny = 1e-300
    for i in range(n):
        off = e[i - 1] ** 2 / q if i > 0 else 0.0
        q = d[i] - x - off
        if q == 0.0:
            q = -tiny
        if q < 0:
            cnt += 1
    return cnt


def jacobi_eig(A, tol=1e-15, max_sweeps=100):
    """Cyclic Jacobi eigen-decomposition of a small real symmetric matrix.
    Returns (w ascending, V) with A V = V diag(w)."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    scale = max(np.abs(A).max(), 1e-300)
    for _ in range(max_sweeps):
        off = np.sqrt(np.sum((A - np.diag(np.diag(A))) ** 2))
        if off <= tol * scale:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if A[p, q] == 0.0:
                    continue
                d = A[q, q] - A[p, p]
                if abs(A[p, q]) <= 1e-150 * abs(d):  # theta would overflow: t = 1/(2 theta) = a_pq/d
                    t = A[p, q] / d
                else:
                    theta = d / (2.0 * A[p, q])
                    t = np.sign(theta) / (abs(theta) + np.hypot(theta, 1.0)) if theta != 0 else 1.0
                c = 1.0 / np.sqrt(t * t + 1.0)
                s = t * c
                R = np.eye(n)
                R[p, p] = c
                R[q, q] = c
                R[p, q] = s
                R[q, p] = -s
                A = R.T @ A @ R
                V = V @ R
    w = np.diag(A).copy()
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]


def real_embedding(M):
    """[[Re M, -Im M], [Im M, Re M]]: each eigenvalue of a Hermitian M appears twice."""
    M = np.asarray(M)
    if not np.iscomplexobj(M):
        return np.array(M, dtype=np.float64)
    R, I = M.real, M.imag
    return np.block([[R, -I], [I, R]])


def herm_from_lower(M):
    M = np.array(M)
    L = np.tril(M)
    return L + np.tril(M, -1).conj().T


def norm1(M):
    return float(np.abs(M).sum(axis=0).max())
