"""CPU model of the one-stage tridiagonalisation scheme of td1.cu (k_td_panel) and of its grouped
back-transform (bt_he2hb with one-stage panels), checked against the FP64 CPU oracle's unblocked
reduction (``oracle.sytrd``) and its reflector-by-reflector back-transform (``oracle.ormtr``).

The model follows the kernel's steps in numpy: per panel of nb columns the trailing block stays as it
was at the panel's start and the panel's reflectors are carried as (V, W); per column the column
update by V, W, the reflector (same convention as the oracle), the Hermitian product with the panel-start
trailing block from its lower triangle only (diagonal real), the rank-2c corrections, w0 = tau p and
w = w0 + alpha v with alpha = -Re(tau w0^H v) / 2; the raw T column (V^H v above the diagonal, tau on
it) finished by the forward recurrence at the panel's end; the rank-2nb trailing update.  The
back-transform merges up to four panels into one compact-WY block whose T comes from the panels' T and
the Gram blocks.  Panel widths 4, 8 and 16 exercise many panels, groups of four and ragged last panels."""
import numpy as np
import pytest

import oracle
from tests.pins import norm1


def herm(n, cx, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cx else 0)
    return (G + G.conj().T) / 2


def lower_hermitian(B):
    """The Hermitian matrix the kernel's tiles see: the lower triangle, mirrored, diagonal real."""
    L = np.tril(B, -1)
    return L + L.conj().T + np.diag(np.diag(B).real)


def td_model(A, nb):
    n = A.shape[0]
    dt = A.dtype
    A = np.array(A, dtype=dt)
    d = np.zeros(n)
    e = np.zeros(max(n - 1, 0))
    V1 = np.zeros((n, n), dtype=dt)
    Ts = []
    for j0 in range(0, n, nb):
        pw = min(nb, n - j0)
        V = np.zeros((n, nb), dtype=dt)
        W = np.zeros((n, nb), dtype=dt)
        T = np.zeros((nb, nb), dtype=dt)
        for c in range(pw):
            j = j0 + c
            col = A[j:, j] - V[j:, :c] @ W[j, :c].conj() - W[j:, :c] @ V[j, :c].conj()
            A[j:, j] = col
            d[j] = col[0].real
            if j == n - 1:
                break
            x = A[j + 1:, j]
            alpha = x[0]
            xn = float(np.sum(np.abs(x[1:]) ** 2))
            if xn == 0.0 and np.imag(alpha) == 0.0:
                beta, tau, scale = float(np.real(alpha)), 0.0, 0.0
            else:
                nrm = np.sqrt(abs(alpha) ** 2 + xn)
                beta = -nrm if np.real(alpha) >= 0 else nrm
                tau = (beta - alpha) / beta
                scale = 1.0 / (alpha - beta)
            e[j] = beta
            v = np.zeros(n, dtype=dt)
            v[j + 1] = 1.0
            v[j + 2:] = scale * x[1:]
            V1[:, j] = v
            V[:, c] = v
            vs = v[j + 1:]
            p = lower_hermitian(A[j + 1:, j + 1:]) @ vs
            vhv = V[j + 1:, :c].conj().T @ vs
            whv = W[j + 1:, :c].conj().T @ vs
            p = p - V[j + 1:, :c] @ whv - W[j + 1:, :c] @ vhv
            w0 = tau * p
            alp = -0.5 * np.real(tau * (w0.conj() @ vs))
            W[j + 1:, c] = w0 + alp * vs
            T[:c, c] = vhv  # raw column: V^H v_c above the diagonal, tau_c on it
            T[c, c] = tau
        nr = min(pw, n - 1 - j0)
        for cc in range(1, nr):
            g = T[:cc, cc].copy()
            for i in range(cc):
                T[i, cc] = -T[cc, cc] * (T[i, i:cc] @ g[i:cc])
        T[nr:, :] = 0
        T[:, nr:] = 0
        Ts.append(T)
        r0 = j0 + nb
        if j0 + pw < n:
            A[r0:, r0:] -= V[r0:] @ W[r0:].conj().T + W[r0:] @ V[r0:].conj().T
    return d, e, V1, Ts


def back_model(V1, Ts, nb, Z, group=4):
    n = V1.shape[0]
    nrefl = n - 1
    npan = (nrefl + nb - 1) // nb if nrefl > 0 else 0
    Y = np.array(Z, dtype=V1.dtype)
    if npan == 0:
        return Y
    G = min(group, npan)
    width = lambda p: min(nb, nrefl - p * nb)
    for q in range((npan + G - 1) // G - 1, -1, -1):
        p0 = q * G
        pc = min(G, npan - p0)
        w = sum(width(p0 + j) for j in range(pc))
        j0 = p0 * nb
        r0 = j0 + 1
        Yg = V1[r0:, j0:j0 + w]
        Tg = np.zeros((w, w), dtype=V1.dtype)
        w0 = width(p0)
        Tg[:w0, :w0] = Ts[p0][:w0, :w0]
        Gg = Yg.conj().T @ Yg
        for j in range(1, pc):
            oj, wj = j * nb, width(p0 + j)
            Tj = Ts[p0 + j][:wj, :wj]
            Tg[:oj, oj:oj + wj] = -Tg[:oj, :oj] @ (Gg[:oj, oj:oj + wj] @ Tj)
            Tg[oj:oj + wj, oj:oj + wj] = Tj
        Y[r0:] -= Yg @ (Tg @ (Yg.conj().T @ Y[r0:]))
    return Y


@pytest.mark.parametrize("nb", [4, 8, 16])
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 40, 70])
def test_panel_scheme_matches_unblocked_reduction(n, cx, nb):
    A = herm(n, cx, 3 + n)
    d, e, V1, Ts = td_model(A, nb)
    do, eo, Vo, tau = oracle.sytrd(A)
    a1 = norm1(A)
    assert np.max(np.abs(d - do)) <= 1e-12 * a1
    if n > 1:
        assert np.max(np.abs(e - eo)) <= 1e-12 * a1
    # each panel's compact-WY block equals the product of its reflectors
    for p, T in enumerate(Ts):
        j0 = p * nb
        nr = min(nb, n - 1 - j0)
        if nr <= 0:
            continue
        Q = np.eye(n, dtype=A.dtype)
        for c in range(nr):
            v = V1[:, j0 + c]
            Q = Q @ (np.eye(n) - T[c, c] * np.outer(v, v.conj()))
        Vp = V1[:, j0:j0 + nr]
        assert np.max(np.abs(Q - (np.eye(n) - Vp @ T[:nr, :nr] @ Vp.conj().T))) <= 1e-13


@pytest.mark.parametrize("nb", [4, 8, 16])
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,k", [(2, 2), (5, 3), (40, 40), (70, 17)])
def test_grouped_back_transform_matches_reflector_by_reflector(n, k, cx, nb):
    A = herm(n, cx, 11 + n)
    d, e, V1, Ts = td_model(A, nb)
    _, _, Vo, tau = oracle.sytrd(A)
    rng = np.random.default_rng(n + k)
    Z = rng.standard_normal((n, k))
    Y = back_model(V1, Ts, nb, Z)
    Yo = oracle.ormtr(Vo, tau, Z.astype(A.dtype))
    assert np.max(np.abs(Y - Yo)) <= 1e-12 * max(1.0, np.abs(Z).max()) * np.sqrt(n)
    # and the back-transformed eigenvectors of T are eigenvectors of A
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    w, Zt = np.linalg.eigh(T)
    Yt = back_model(V1, Ts, nb, Zt)
    assert np.max(np.abs(A @ Yt - Yt * w)) <= 1e-12 * norm1(A)
