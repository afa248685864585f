"""FP64 CPU oracle for  H C = S C Lambda  (Eq. 2): ctypes wrapper over ``oracle_gev.c``.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py``.  The GPU solver package never imports this module, and this module imports
nothing from it.

Every function takes and returns numpy arrays.  Matrices are passed column-major (Fortran order);
only the lower triangles of H and S are read.  Real inputs use the ``oracle_d_*`` symbols, complex
inputs (complex128) the ``oracle_z_*`` symbols.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_gev.so")
_SRC = os.path.join(_HERE, "oracle_gev.c")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (real and complex objects in one shared library)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    flags = ["-O2", "-fPIC", "-fopenmp", "-std=c11"]
    objs = []
    for tag, defs in (("d", []), ("z", ["-DORACLE_COMPLEX"])):
        obj = os.path.join(_BUILD, f"oracle_{tag}.o")
        subprocess.check_call(["gcc", *flags, *defs, "-c", _SRC, "-o", obj])
        objs.append(obj)
    tmp = _LIB_PATH + ".tmp"
    subprocess.check_call(["gcc", "-shared", "-fopenmp", "-o", tmp, *objs, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.c_void_p
        i = ctypes.c_int
        for p in ("d", "z"):
            getattr(_lib, f"oracle_{p}_potrf").argtypes = [i, dp, i]
            getattr(_lib, f"oracle_{p}_potrf").restype = i
            getattr(_lib, f"oracle_{p}_reduce").argtypes = [i, dp, i, dp, i, dp, i, dp]
            getattr(_lib, f"oracle_{p}_sytrd").argtypes = [i, dp, i, dp, dp, dp]
            getattr(_lib, f"oracle_{p}_ormtr").argtypes = [i, i, dp, i, dp, dp, i]
            getattr(_lib, f"oracle_{p}_normalize_phase").argtypes = [i, i, dp, i]
            getattr(_lib, f"oracle_{p}_check").argtypes = [i, i, dp, i, dp, i, dp, dp, i, dp, dp]
            getattr(_lib, f"oracle_{p}_gev").argtypes = [i, dp, i, dp, i, i, dp, dp, i, dp]
            getattr(_lib, f"oracle_{p}_gev").restype = i
            getattr(_lib, f"oracle_{p}_density").argtypes = [i, i, dp, i, dp, dp, i]
            getattr(_lib, f"oracle_{p}_density").restype = None
            getattr(_lib, f"oracle_{p}_gev_reduced").argtypes = [i, dp, i, dp, i, ctypes.c_double, i, dp, dp, i,
                                                                   dp]
            getattr(_lib, f"oracle_{p}_gev_reduced").restype = i
        _lib.oracle_d_steql.argtypes = [i, dp, dp, dp, dp, i]
        _lib.oracle_d_steql.restype = i
    return _lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _prefix(a: np.ndarray) -> str:
    return "z" if np.iscomplexobj(a) else "d"


def _fortran(a: np.ndarray, complex_: bool) -> np.ndarray:
    return np.asfortranarray(a, dtype=np.complex128 if complex_ else np.float64)


def potrf(S: np.ndarray):
    """Unblocked Cholesky of the lower triangle (reduction step 1).  Returns (L, info)."""
    cx = np.iscomplexobj(S)
    L = _fortran(np.array(S), cx).copy(order="F")
    n = L.shape[0]
    info = getattr(lib(), f"oracle_{_prefix(L)}_potrf")(n, _ptr(L), n)
    return L, int(info)


def reduce(H: np.ndarray, L: np.ndarray):
    """A = L^{-1} H L^{-H} by forward substitutions (reduction steps 2-3).  Returns (A, asym)."""
    cx = np.iscomplexobj(H) or np.iscomplexobj(L)
    H = _fortran(H, cx)
    L = _fortran(L, cx)
    n = H.shape[0]
    A = np.zeros((n, n), dtype=H.dtype, order="F")
    asym = np.zeros(1)
    getattr(lib(), f"oracle_{_prefix(H)}_reduce")(n, _ptr(H), n, _ptr(L), n, _ptr(A), n, _ptr(asym))
    return A, float(asym[0])


def sytrd(A: np.ndarray):
    """One-stage Householder tridiagonalisation of a full Hermitian A.  Returns (d, e, V, tau)
    where V holds the reflectors below the subdiagonal (as stored by the oracle)."""
    cx = np.iscomplexobj(A)
    V = _fortran(np.array(A), cx).copy(order="F")
    n = V.shape[0]
    d = np.zeros(n)
    e = np.zeros(max(n, 1))
    tau = np.zeros(max(n, 1), dtype=V.dtype)
    getattr(lib(), f"oracle_{_prefix(V)}_sytrd")(n, _ptr(V), n, _ptr(d), _ptr(e), _ptr(tau))
    return d, e[: max(n - 1, 0)].copy(), V, tau


def ormtr(V: np.ndarray, tau: np.ndarray, Z: np.ndarray):
    """Y = Q Z with Q the product of the reflectors returned by :func:`sytrd`."""
    cx = np.iscomplexobj(V)
    Y = _fortran(np.array(Z), cx).copy(order="F")
    n, k = Y.shape
    getattr(lib(), f"oracle_{_prefix(V)}_ormtr")(n, k, _ptr(V), n, _ptr(tau), _ptr(Y), n)
    return Y


def steql(d: np.ndarray, e: np.ndarray):
    """Implicit-QL eigen-solve of the real symmetric tridiagonal (d, e).  Returns (w, Z, status)."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = d.shape[0]
    e = np.ascontiguousarray(np.concatenate([np.asarray(e, dtype=np.float64), [0.0]]))
    w = np.zeros(n)
    Z = np.zeros((n, n), order="F")
    st = lib().oracle_d_steql(n, _ptr(d), _ptr(e), _ptr(w), _ptr(Z), n)
    return w, Z, int(st)


def check(H, S, w, C):
    """Residual ||HC - SC diag(w)||_1/(||H||_1 ||C||_1) and orthogonality ||C^H S C - I||_1."""
    cx = np.iscomplexobj(H) or np.iscomplexobj(C)
    H = _fortran(H, cx)
    S = _fortran(S, cx)
    C = _fortran(C, cx)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n, k = C.shape
    r = np.zeros(1)
    o = np.zeros(1)
    getattr(lib(), f"oracle_{_prefix(H)}_check")(n, k, _ptr(H), n, _ptr(S), n, _ptr(w), _ptr(C), n,
                                                   _ptr(r), _ptr(o))
    return float(r[0]), float(o[0])


def normalize_phase(C: np.ndarray) -> np.ndarray:
    cx = np.iscomplexobj(C)
    C = _fortran(np.array(C), cx).copy(order="F")
    n, k = C.shape
    getattr(lib(), f"oracle_{_prefix(C)}_normalize_phase")(n, k, _ptr(C), n)
    return C


def density(C: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Full n x n P with P_ij = sum_l g_l conj(C_il) C_jl (section "Circumventing the eigenvalue
    problem"; g = occupation numbers f, or f * lambda for the energy-weighted matrix)."""
    cx = np.iscomplexobj(C)
    C = _fortran(C, cx)
    n, k = C.shape
    g = np.ascontiguousarray(np.broadcast_to(np.asarray(g, dtype=np.float64), (k,)))
    P = np.zeros((n, n), dtype=C.dtype, order="F")
    getattr(lib(), f"oracle_{_prefix(C)}_density")(n, k, _ptr(C), n, _ptr(g), _ptr(P), n)
    return P


def gev(H: np.ndarray, S: np.ndarray, k: int):
    """The k lowest eigenpairs of the pencil (H, S).

    Returns ``(w, C, info, diag)``: eigenvalues ascending, S-orthonormal eigenvectors (phase
    normalised), status (0 ok, p+1 > 0 non-positive pivot p, -1 no QL convergence, -2 bad
    arguments) and ``diag = {resid, ortho, asym}``.
    """
    cx = np.iscomplexobj(H) or np.iscomplexobj(S)
    H = _fortran(H, cx)
    S = _fortran(S, cx)
    n = H.shape[0]
    w = np.zeros(max(k, 1))
    C = np.zeros((n, max(k, 1)), dtype=H.dtype, order="F")
    dg = np.zeros(4)
    info = getattr(lib(), f"oracle_{_prefix(H)}_gev")(n, _ptr(H), n, _ptr(S), n, k, _ptr(w), _ptr(C),
                                                       max(n, 1), _ptr(dg))
    return w[:k].copy(), C[:, :k].copy(order="F"), int(info), {
        "resid": float(dg[0]), "ortho": float(dg[1]), "asym": float(dg[2])}


def gev_reduced(H: np.ndarray, S: np.ndarray, delta: float, k: int):
    """The k lowest eigenpairs of (H, S) in the basis of the eigenvectors of S with eigenvalue
    >= delta (the procedure for an ill-conditioned S, section "Current Status of the
    Implementation").  Returns ``(w, C, m, status)``: eigenvalues ascending, C = X Y (n x k, phase
    normalised), the kept basis size m, status (0 ok, -1 no QL convergence, -2 bad arguments,
    -3 k > m)."""
    cx = np.iscomplexobj(H) or np.iscomplexobj(S)
    H = _fortran(H, cx)
    S = _fortran(S, cx)
    n = H.shape[0]
    w = np.zeros(max(k, 1))
    C = np.zeros((n, max(k, 1)), dtype=H.dtype, order="F")
    m = np.zeros(1, dtype=np.int32)
    st = getattr(lib(), f"oracle_{_prefix(H)}_gev_reduced")(n, _ptr(H), n, _ptr(S), n, float(delta), k, _ptr(w),
                                                            _ptr(C), max(n, 1), _ptr(m))
    return w[:k].copy(), C[:, :k].copy(order="F"), int(m[0]), int(st)
