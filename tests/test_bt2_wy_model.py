"""CPU model of back-transform 2 in compact-WY form (the scheme of bt_levels_wy in bulge.cu and the
block-diagonal product mode of ozaki.cu / tc_gemm.cu), checked against the reflector-by-reflector
application of the same reflector store.

Reflector store: sweep s, task t has v (v_0 = 1, length b) acting on rows s + 1 + t b ...; a task that
never ran has tau = 0 and arbitrary (here: huge) entries that must not reach the result.  Level L
holds the blocks D_j = H(s0) ... H(s0 + b - 1) (group g = s0 / b, task t = L - (ngroups - 1 - g)); the
model forms T_j by the forward recurrence, W_j = V_j T_j, and applies
P = blockdiag(V_j^H) Y_L, Y_L -= blockdiag(W_j) P.  It also checks that each 128-row tile's compact K
range (bd_range) holds every non-zero of the block-diagonal operands."""
import numpy as np
import pytest

OM, KS = 128, 16


def bd_range(bm, bk, mt):
    if bm <= OM:
        per = OM // bm
        return mt * per * bk // KS, per * bk // KS
    return (mt // (bm // OM)) * bk // KS, bk // KS


def level_blocks(n, b, L, ngroups, ntask):
    g_lo = max(0, ngroups - 1 - L)
    g_hi = min(ngroups - 1, ntask - 1 + ngroups - 1 - L)
    w0 = lambda g: (2 * g + L - ngroups + 1) * b + 1
    while g_hi >= g_lo and w0(g_hi) >= n:
        g_hi -= 1
    if g_hi < g_lo:
        return None
    return g_lo, g_hi - g_lo + 1, w0(g_lo)


def store(n, b, cx, rng):
    ntask = (n + b - 1) // b + 2
    V2 = rng.standard_normal((n * ntask, b)) + (1j * rng.standard_normal((n * ntask, b)) if cx else 0)
    V2[:, 0] = 1.0
    tau2 = np.zeros(n * ntask, dtype=complex if cx else float)
    for sw in range(n):
        for t in range(ntask):
            p = sw + 1 + t * b
            ln = min(b, n - p) if p < n else 0
            rid = sw * ntask + t
            if sw > n - 3 or ln <= 1:
                V2[rid, 1:] = 1e300  # never used: tau = 0
                continue
            V2[rid, ln:] = 0
            tau2[rid] = 2.0 / np.sum(np.abs(V2[rid]) ** 2)
    return V2, tau2, ntask


def sequential(n, b, V2, tau2, ntask, Y):
    ngroups = (n - 3) // b + 1
    for L in range(ngroups + ntask):
        for g in range(max(0, ngroups - 1 - L), ngroups):
            t = L - (ngroups - 1 - g)
            if t < 0 or t >= ntask:
                continue
            s0, s1 = g * b, min(g * b + b - 1, n - 3)
            if s0 + 1 + t * b >= n:
                continue
            for q in range(s1 - s0, -1, -1):
                tau = tau2[(s0 + q) * ntask + t]
                if tau == 0:
                    continue
                p = s0 + q + 1 + t * b
                ln = min(b, n - p)
                v = V2[(s0 + q) * ntask + t, :ln]
                Y[p:p + ln] -= np.outer(v, tau * (v.conj() @ Y[p:p + ln]))
    return Y


def wy_levels(n, b, V2, tau2, ntask, Y):
    ngroups = (n - 3) // b + 1
    dt = Y.dtype
    for L in range(ngroups + ntask):
        lb = level_blocks(n, b, L, ngroups, ntask)
        if lb is None:
            continue
        g_lo, nblk, w00 = lb
        rows = min(nblk * 2 * b, n - w00)
        A1 = np.zeros((nblk * b, rows), dtype=dt)
        A2 = np.zeros((rows, nblk * b), dtype=dt)
        for j in range(nblk):
            g = g_lo + j
            t = L - (ngroups - 1 - g)
            Vs = np.zeros((2 * b, b), dtype=dt)
            taus = np.zeros(b, dtype=dt)
            for q in range(b):
                sw = g * b + q
                if sw > n - 3 or tau2[sw * ntask + t] == 0:
                    continue
                taus[q] = tau2[sw * ntask + t]
                for r in range(q, q + b):
                    if w00 + 2 * b * j + r < n:
                        Vs[r, q] = V2[sw * ntask + t, r - q]
            T = np.zeros((b, b), dtype=dt)
            for q in range(b):
                T[:q, q] = -taus[q] * (T[:q, :q] @ (Vs[:, :q].conj().T @ Vs[:, q]))
                T[q, q] = taus[q]
            W = Vs @ T
            for r in range(min(2 * b, rows - 2 * b * j)):
                A1[j * b:(j + 1) * b, 2 * b * j + r] = Vs[r].conj()
                A2[2 * b * j + r, j * b:(j + 1) * b] = W[r]
        for A, bm, bk in ((A1, b, 2 * b), (A2, 2 * b, b)):
            for i in range(A.shape[0]):
                f, c = bd_range(bm, bk, i // OM)
                nz = np.nonzero(A[i])[0]
                assert nz.size == 0 or (nz.min() >= f * KS and nz.max() < (f + c) * KS)
        Yl = Y[w00:w00 + rows]
        Yl -= A2 @ (A1 @ Yl)
    return Y


@pytest.mark.parametrize("n,b,k,cx", [(3, 16, 2, False), (40, 16, 7, False), (131, 16, 9, True),
                                      (200, 32, 5, False), (300, 64, 6, True), (261, 64, 4, False)])
def test_wy_levels_match_sequential_reflectors(n, b, k, cx):
    rng = np.random.default_rng(n + b)
    V2, tau2, ntask = store(n, b, cx, rng)
    Y0 = rng.standard_normal((n, k)) + (1j * rng.standard_normal((n, k)) if cx else 0)
    Ys = sequential(n, b, V2, tau2, ntask, Y0.copy())
    Yw = wy_levels(n, b, V2, tau2, ntask, Y0.copy())
    assert np.all(np.isfinite(Yw))
    assert np.max(np.abs(Yw - Ys)) <= 1e-13 * np.max(np.abs(Ys))
