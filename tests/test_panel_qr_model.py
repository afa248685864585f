"""CPU model of the single-barrier Householder panel factorisation of sbr.cu (k_panel_qr), checked
against numpy's QR and against the definition of the compact-WY factor.

Per column c the kernel's blocks sum, over their rows strictly below the pivot and with the UNSCALED
column x: ||x||^2, u_j = sum conj(x_r) P(r, j) for the columns still to update (j > c) and
t_j = sum conj(P(r, j)) x_r for the stored reflectors (j < c); then, from those sums alone, the reflector
(beta = -sign(Re alpha) ||(alpha, x)||, tau = (beta - alpha) / beta, v = (1, x / (alpha - beta))) and the
exact inner products
    w_j = v^H P(:, j) = P(c, j) + conj(scale) u_j,     s_j = Y(:, j)^H v = conj(P(c, j)) + scale t_j,
which give the update P(:, j) -= v conj(tau) w_j and the column T(0:c, c) = -tau T(0:c, 0:c) s.  The model
runs exactly these steps in numpy."""
import numpy as np
import pytest


def panel_qr_model(P):
    P = np.array(P)
    m, b = P.shape
    Y = np.zeros_like(P)
    T = np.zeros((b, b), dtype=P.dtype)
    for c in range(b):
        if c >= m:
            continue
        x = P[c + 1:, c]
        xn = float(np.sum(np.abs(x) ** 2))
        u = np.array([np.sum(np.conj(x) * P[c + 1:, j]) if j > c else 0 for j in range(b)], dtype=P.dtype)
        t = np.array([np.sum(np.conj(P[c + 1:, j]) * x) if j < c else 0 for j in range(b)], dtype=P.dtype)
        alpha = P[c, c]
        if xn == 0.0 and np.imag(alpha) == 0.0:
            continue  # trivial reflector: T column zero, P unchanged
        nrm = np.sqrt(abs(alpha) ** 2 + xn)
        beta = -nrm if np.real(alpha) >= 0 else nrm
        tau = (beta - alpha) / beta
        scale = 1.0 / (alpha - beta)
        pc = P[c, :].copy()
        w = pc + np.conj(scale) * u
        s = np.conj(pc) + scale * t
        P[c + 1:, c] = scale * x
        P[c, c] = beta
        v = np.concatenate([[1.0], P[c + 1:, c]])
        for j in range(c + 1, b):
            P[c:, j] -= v * (np.conj(tau) * w[j])
        T[:c, c] = -tau * (T[:c, :c] @ s[:c])
        T[c, c] = tau
        # (the stored reflectors of later columns read their own column below the pivot)
    for j in range(b):
        if j < m:
            Y[j, j] = 1.0
            Y[j + 1:, j] = P[j + 1:, j]
    R = np.triu(P[:b, :]) if m >= b else np.triu(P)
    return Y, T, R


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("m,b", [(1, 1), (3, 4), (16, 16), (40, 16), (100, 32), (70, 64)])
def test_panel_model_is_a_householder_qr(m, b, cx):
    rng = np.random.default_rng(m + 7 * b)
    P0 = rng.standard_normal((m, b)) + (1j * rng.standard_normal((m, b)) if cx else 0)
    Y, T, R = panel_qr_model(P0)
    Q = np.eye(m) - Y @ T @ Y.conj().T
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(m))) <= 1e-13
    QhP = Q.conj().T @ P0
    k = min(m, b)
    assert np.max(np.abs(np.tril(QhP, -1))) <= 1e-12 * np.abs(P0).max() * m
    assert np.max(np.abs(QhP[:k] - R[:k])) <= 1e-12 * np.abs(P0).max() * m
    Rn = np.linalg.qr(P0, mode="r")
    assert np.allclose(np.abs(np.diag(R[:k, :k])), np.abs(np.diag(Rn[:k, :k])), rtol=1e-12, atol=1e-12)
    # the reflectors' convention: real diagonal of R, opposite in sign to Re of the pivot it replaced
    assert np.max(np.abs(np.imag(np.diag(R[:k, :k])))) == 0.0


def test_trivial_column_keeps_a_zero_reflector():
    P0 = np.zeros((5, 2))
    P0[0, 0] = 3.0
    P0[:, 1] = np.arange(5.0)
    Y, T, R = panel_qr_model(P0)
    assert T[0, 0] == 0.0 and R[0, 0] == 3.0
    Q = np.eye(5) - Y @ T @ Y.T
    assert np.max(np.abs(np.tril(Q.T @ P0, -1))) <= 1e-13
