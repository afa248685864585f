"""Seeded synthetic inputs for  H C = S C Lambda  (Eq. 2), shared by the oracle tests and the GPU path.

This module builds test problems only; it contains none of the solver's arithmetic.

Recipe (DFT-like pencils standing in for the FHI-aims matrices of Table 1, which are not public):

* overlap S: Hermitian Toeplitz
    real    S_ij = exp(-0.5 |i-j|) cos(0.3 |i-j|) + 0.05 delta_ij
    complex S_ij = exp(-0.4 |i-j|) exp(i 0.2 (i-j)) + 0.02 delta_ij
* spectrum lambda: 10 % "core" U[-100,-10], 40 % "valence" U[-1,0], the rest "conduction" U[0,5],
  drawn in that order with ``numpy.random.default_rng(seed)``; counts round(0.1 N), round(0.4 N).
* Q: Haar orthogonal/unitary, QR of a Gaussian matrix (complex: (g1 + i g2)/sqrt 2) with the column
  phases fixed by diag(R).
* H = S^{1/2} Q diag(lambda) Q^H S^{1/2} with S^{1/2} the Hermitian square root, so that
  S^{-1/2} H S^{-1/2} = Q diag(lambda) Q^H and the generalized eigenvalues are exactly lambda.
* optional near-degenerate cluster: the 16 sorted eigenvalues at [k/2, k/2+16) are replaced by
  c + 1e-8 j/15 (j = 0..15), c the first of them.

``make_problem`` returns numpy arrays in Fortran (column-major) order, or torch tensors holding the
same column-major data when ``device`` is given (the dense linear algebra of the construction then
runs through torch on that device, which is much faster at N >= 8192).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Problem:
    n: int
    k: int
    seed: int
    complex: bool
    H: object  # numpy (Fortran order) or torch tensor (column-major data, see module docstring)
    S: object
    lam: np.ndarray  # the exact generalized eigenvalues, ascending (length n)
    note: str = ""


def overlap_toeplitz(n: int, complex_: bool) -> np.ndarray:
    i = np.arange(n)
    diff = i[:, None] - i[None, :]
    ad = np.abs(diff).astype(np.float64)
    if complex_:
        S = np.exp(-0.4 * ad) * np.exp(1j * 0.2 * diff) + 0.02 * np.eye(n)
    else:
        S = np.exp(-0.5 * ad) * np.cos(0.3 * ad) + 0.05 * np.eye(n)
    return np.asfortranarray(S)


def draw_spectrum(n: int, rng: np.random.Generator) -> np.ndarray:
    n_core = int(round(0.1 * n))
    n_val = int(round(0.4 * n))
    n_cond = n - n_core - n_val
    core = rng.uniform(-100.0, -10.0, n_core)
    val = rng.uniform(-1.0, 0.0, n_val)
    cond = rng.uniform(0.0, 5.0, n_cond)
    return np.concatenate([core, val, cond])


def insert_cluster(lam_sorted: np.ndarray, k: int, size: int = 16, width: float = 1e-8) -> np.ndarray:
    lam = lam_sorted.copy()
    a = k // 2
    c = lam[a]
    lam[a:a + size] = c + width * np.arange(size) / (size - 1)
    return np.sort(lam, kind="stable")


def gaussian(n: int, rng: np.random.Generator, complex_: bool) -> np.ndarray:
    if complex_:
        g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        return g / math.sqrt(2.0)
    return rng.standard_normal((n, n))


def _build_numpy(S, lam, G):
    Q, R = np.linalg.qr(G)
    dr = np.diag(R)
    ph = dr / np.abs(dr)
    Q = Q * ph[None, :]
    sig, V = np.linalg.eigh(S)
    Sh = (V * np.sqrt(sig)[None, :]) @ V.conj().T
    Sh = 0.5 * (Sh + Sh.conj().T)
    M = (Q * lam[None, :]) @ Q.conj().T
    H = Sh @ M @ Sh
    H = 0.5 * (H + H.conj().T)
    return np.asfortranarray(H)


def _build_torch(S, lam, G, device):
    import torch

    St = torch.from_numpy(np.ascontiguousarray(S)).to(device)
    Gt = torch.from_numpy(np.ascontiguousarray(G)).to(device)
    del G
    Q, R = torch.linalg.qr(Gt)
    del Gt
    dr = torch.diagonal(R)
    Q = Q * (dr / dr.abs())[None, :]
    del R
    sig, V = torch.linalg.eigh(St)
    Sh = (V * sig.sqrt().to(V.dtype)[None, :]) @ V.conj().transpose(0, 1)
    Sh = 0.5 * (Sh + Sh.conj().transpose(0, 1))
    del V
    lt = torch.from_numpy(lam).to(device).to(Q.dtype)
    M = (Q * lt[None, :]) @ Q.conj().transpose(0, 1)
    del Q
    H = Sh @ M @ Sh
    del M, Sh
    H = 0.5 * (H + H.conj().transpose(0, 1))
    # column-major data: the row-major buffer of H^T
    Hc = H.transpose(0, 1).contiguous()
    Sc = St.transpose(0, 1).contiguous()
    return Hc, Sc


def make_problem(n: int, k: int, seed: int, complex_: bool = False, cluster: bool = False,
                 device=None, gap_check: bool = True) -> Problem:
    """Build the seeded pencil (H, S) of size n with exact eigenvalues; see the module docstring."""
    note = ""
    cur_seed = seed
    for _attempt in range(8):
        rng = np.random.default_rng(cur_seed)
        lam = np.sort(draw_spectrum(n, rng), kind="stable")
        if cluster:
            lam = insert_cluster(lam, k)
        S = overlap_toeplitz(n, complex_)
        G = gaussian(n, rng, complex_)
        if device is None:
            H = _build_numpy(S, lam, G)
            Hn = H
        else:
            H, S = _build_torch(S, lam, G, device)
            Hn = None
        del G
        if gap_check and cluster and k < n:
            if Hn is not None:
                h1 = float(np.abs(Hn).sum(axis=0).max())
            else:
                h1 = float(H.abs().sum(dim=1).max().item())
            if not (lam[k] - lam[k - 1] > 1e-6 * h1):
                cur_seed += 1000
                note = f"redrawn with seed {cur_seed} (gap at k too small)"
                continue
        return Problem(n, k, cur_seed, complex_, H, S, lam, note)
    raise RuntimeError("could not draw a pencil with a spectral gap at k")


def lower_only(M: np.ndarray, garbage: float | None = None) -> np.ndarray:
    """Copy of M with the strict upper triangle replaced (by NaN or a value): checks that a solver
    reads the lower triangle only."""
    out = np.array(M, order="F", copy=True)
    iu = np.triu_indices(out.shape[0], 1)
    out[iu] = np.nan if garbage is None else garbage
    return out


def tridiag_toeplitz(n: int):
    """tridiag(-1, 2, -1) with eigenvalues 2 - 2 cos(j pi/(n+1)), j = 1..n."""
    return 2.0 * np.ones(n), -np.ones(max(n - 1, 0))


def random_tridiag(n: int, seed: int):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n), rng.standard_normal(max(n - 1, 0))


def glued_wilkinson(m: int, copies: int, glue: float):
    """Wilkinson W_m^+ blocks glued by small off-diagonals: a classic hard case for deflation."""
    h = (m - 1) / 2.0
    blk = np.abs(np.arange(m) - h)
    d = np.concatenate([blk] * copies)
    e = np.ones(m * copies - 1)
    for c in range(1, copies):
        e[c * m - 1] = glue
    return d, e


def singular_overlap_pencil(n: int, m: int, complex_: bool, seed: int, dropped=(1e-9, 1e-12, 0.0)):
    """A pencil with a numerically singular overlap: S = U diag(sigma) U^H with n - m eigenvalues from
    ``dropped`` (below any usual threshold delta) and m drawn from U[0.1, 3];
    H = U_m sigma_m^{1/2} Q diag(lambda) Q^H sigma_m^{1/2} U_m^H + U_d G U_d^H with lambda ~ U[-10, 5]
    (sorted), Q Haar on the kept space and an arbitrary Hermitian G on the dropped directions.  In the
    eigenbasis of S restricted to the kept directions the pencil's eigenvalues are exactly lambda.
    Returns (H, S, lambda, U_d) as numpy arrays (Fortran order)."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(gaussian(n, rng, complex_))
    sig = np.concatenate([np.resize(np.array(dropped, dtype=np.float64), n - m), rng.uniform(0.1, 3.0, m)])
    S = (U * sig[None, :]) @ U.conj().T
    S = 0.5 * (S + S.conj().T)
    lam = np.sort(rng.uniform(-10.0, 5.0, m))
    Q, _ = np.linalg.qr(gaussian(m, rng, complex_))
    Um, Ud = U[:, n - m:], U[:, : n - m]
    sh = np.sqrt(sig[n - m:])
    Hm = (Um * sh[None, :]) @ ((Q * lam[None, :]) @ Q.conj().T) @ (Um * sh[None, :]).conj().T
    Gd = gaussian(n - m, rng, complex_)
    H = Hm + Ud @ (0.5 * (Gd + Gd.conj().T)) @ Ud.conj().T
    H = 0.5 * (H + H.conj().T)
    return np.asfortranarray(H), np.asfortranarray(S), lam, Ud
