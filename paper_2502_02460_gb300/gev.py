"""Thin Python binding of the C ABI in ``include/gev.h`` / ``include/gev_steps.h``.

Argument marshalling only: every step of the solve runs in the CUDA kernels of ``libgev.so``.
PyTorch supplies device memory and the stream.  There is no CPU fallback: if the library is not
built, or no CUDA device is present, the calls raise.

Layout convention.  The library works on column-major matrices.  A column-major ``rows x cols``
matrix M is held here as a contiguous torch tensor of shape ``(cols, rows)`` (the row-major buffer
of M^T); ``cm(M)`` makes one from a logical tensor and ``logical(B)`` views it back.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgev.so")

GEV_F64, GEV_C128 = 0, 1
GEV_PLAIN, GEV_MIXED = 0, 1
ERRORS = {
    1: "GEV_ERR_NOT_SPD", 2: "GEV_ERR_NO_CONVERGENCE", 3: "GEV_ERR_TIMEOUT", 4: "GEV_ERR_OOM",
    5: "GEV_ERR_CUDA", 6: "GEV_ERR_REUSE_WITHOUT_FACTOR", 7: "GEV_ERR_UNSUPPORTED", 9: "GEV_ERR_RANK",
}
STEP_NAMES = ["cholesky", "invert", "multiply", "to_band", "to_tridiag", "solve", "back_tridiag",
              "back_band", "mult", "refine"]
NSTEPS = len(STEP_NAMES)

SYMBOLS = [
    "gev_default_opts", "gev_setup", "gev_solve", "gev_reuse_factor", "gev_free",
    "gev_workspace_bytes", "gev_strerror", "gev_step_potrf", "gev_step_trtri", "gev_step_hegst",
    "gev_step_he2hb", "gev_step_hb2st", "gev_step_stedc", "gev_step_back", "gev_step_mult",
    "gev_density", "gev_check", "gev_solve_reduced", "gev_step_he2td",
]


class GevError(RuntimeError):
    def __init__(self, code: int, where: str, info: int = 0):
        name = ERRORS.get(code, "invalid argument %d" % (-code) if code < 0 else f"error {code}")
        super().__init__(f"{where}: {name}" + (f" (info={info})" if info else ""))
        self.code = code
        self.info = info


class Opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("prec", ctypes.c_int),
                ("band_b", ctypes.c_int), ("panel_nb", ctypes.c_int), ("refine_tol", ctypes.c_double),
                ("refine_max_iter", ctypes.c_int), ("workspace_limit", ctypes.c_size_t),
                ("timing", ctypes.c_int), ("fp64_emulation", ctypes.c_int),
                ("refine_rr_only", ctypes.c_int), ("fp32_products", ctypes.c_int),
                ("wait_limit", ctypes.c_int), ("check", ctypes.c_int), ("debug_stall", ctypes.c_int),
                ("rr_band_b", ctypes.c_int), ("one_stage", ctypes.c_int),
                ("rr_one_stage", ctypes.c_int)]


class Report(ctypes.Structure):
    _fields_ = [("info", ctypes.c_int), ("deflated", ctypes.c_int), ("refine_iters", ctypes.c_int),
                ("reused_factor", ctypes.c_int), ("refine_resid", ctypes.c_double),
                ("ms", ctypes.c_double * NSTEPS), ("workspace_bytes", ctypes.c_size_t),
                ("launches", ctypes.c_longlong), ("gemm_calls", ctypes.c_int),
                ("gemm_ms", ctypes.c_double), ("gemm_flops", ctypes.c_double),
                ("refine_oa_steps", ctypes.c_int), ("resid", ctypes.c_double), ("ortho", ctypes.c_double)]

    def as_dict(self):
        return {"info": self.info, "deflated": self.deflated, "refine_iters": self.refine_iters,
                "reused_factor": self.reused_factor, "refine_resid": self.refine_resid,
                "ms": dict(zip(STEP_NAMES, list(self.ms))), "workspace_bytes": self.workspace_bytes,
                "launches": self.launches, "gemm_calls": self.gemm_calls, "gemm_ms": self.gemm_ms,
                "gemm_flops": self.gemm_flops, "refine_oa_steps": self.refine_oa_steps,
                "resid": self.resid, "ortho": self.ortho}


_lib = None


def lib() -> ctypes.CDLL:
    """Load libgev.so (built by ``paper_2502_02460_gb300.build.build()``); raise if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2502_02460_gb300.build.build() "
                               "(the solver has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        ip = ctypes.POINTER(ctypes.c_int)
        L.gev_default_opts.argtypes = [ctypes.POINTER(Opts)]
        L.gev_default_opts.restype = None
        L.gev_setup.argtypes = [ctypes.POINTER(vp), i, i, ctypes.POINTER(Opts)]
        L.gev_solve.argtypes = [vp, vp, i, vp, i, i, vp, vp, i, ctypes.POINTER(Report)]
        L.gev_reuse_factor.argtypes = [vp, i]
        L.gev_free.argtypes = [vp]
        L.gev_workspace_bytes.argtypes = [i, i, ctypes.POINTER(Opts)]
        L.gev_workspace_bytes.restype = ctypes.c_size_t
        L.gev_strerror.argtypes = [i]
        L.gev_strerror.restype = ctypes.c_char_p
        L.gev_step_potrf.argtypes = [vp, vp, i, ip]
        L.gev_step_trtri.argtypes = [vp, vp, i]
        L.gev_step_hegst.argtypes = [vp, vp, i, vp, i, vp, i]
        L.gev_step_he2hb.argtypes = [vp, vp, i, i, ip]
        L.gev_step_he2td.argtypes = [vp, vp, i, vp, vp]
        L.gev_step_hb2st.argtypes = [vp, vp, vp]
        L.gev_step_stedc.argtypes = [vp, vp, vp, i, vp, vp, i, ip]
        L.gev_step_back.argtypes = [vp, vp, i, i, vp, i]
        L.gev_step_mult.argtypes = [vp, vp, i, vp, i, i, vp, i]
        L.gev_density.argtypes = [vp, i, vp, i, vp, vp, vp, i, vp, i]
        dpp = ctypes.POINTER(ctypes.c_double)
        L.gev_check.argtypes = [vp, vp, i, vp, i, i, vp, vp, i, dpp, dpp]
        L.gev_solve_reduced.argtypes = [vp, vp, i, vp, i, d, i, vp, vp, i, ip, ctypes.POINTER(Report)]
        for s in SYMBOLS:
            getattr(L, s).restype = getattr(L, s).restype or ctypes.c_int
        _lib = L
    return _lib


# ------------------------------------------------------------------------------ layout helpers --
def cm(M):
    """Column-major buffer of a logical torch matrix (shape (cols, rows), contiguous)."""
    return M.transpose(0, 1).contiguous()


def logical(B):
    """Logical matrix view of a column-major buffer."""
    return B.transpose(0, 1)


def cm_from_numpy(M: np.ndarray, device):
    """Column-major device buffer from a numpy matrix."""
    import torch

    return torch.from_numpy(np.ascontiguousarray(np.asarray(M).T)).to(device)


def numpy_from_cm(B) -> np.ndarray:
    """numpy (Fortran-ordered) matrix from a column-major device buffer."""
    return B.detach().cpu().numpy().T


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check(code: int, where: str, info: int = 0):
    if code != 0:
        raise GevError(code, where, info)


# ------------------------------------------------------------------------------------- handle --
class Solver:
    """One handle (``gev_setup``) for problems of order n: workspace, resident factor, stream."""

    def __init__(self, n: int, complex_: bool = False, device=None, mixed: bool = False,
                 band_b: int = 0, panel_nb: int = 0, timing: int = 0, stream=None,
                 workspace_limit: int = 0, refine_tol: float = 0.0, refine_max_iter: int = 0,
                 fp64_emulation: int = -1, refine_rr_only: int = 0, fp32_products: int = -1,
                 wait_limit: int = 0, check: bool = False, debug_stall: bool = False, rr_band_b: int = 0,
                 one_stage=None, rr_one_stage=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the solver needs a CUDA device (no CPU fallback)")
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.n = n
        self.complex = complex_
        self.dtype = torch.complex128 if complex_ else torch.float64
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        o = Opts()
        lib().gev_default_opts(ctypes.byref(o))
        o.device = self.device.index
        o.cuda_stream = ctypes.c_void_p(self.stream.cuda_stream)
        o.prec = GEV_MIXED if mixed else GEV_PLAIN
        if band_b == 0:  # the autotuner's table (tune.py) for this dtype, precision and order
            from . import tune

            band_b = tune.pick_band(n, complex_, mixed)
        self.band_b = band_b
        o.band_b = band_b
        o.panel_nb = panel_nb
        o.timing = int(timing)
        o.workspace_limit = workspace_limit
        o.refine_tol = refine_tol
        o.refine_max_iter = refine_max_iter
        o.fp64_emulation = fp64_emulation
        o.refine_rr_only = refine_rr_only
        o.fp32_products = fp32_products
        o.wait_limit = int(wait_limit)
        o.check = 1 if check else 0
        o.debug_stall = 1 if debug_stall else 0
        o.rr_band_b = int(rr_band_b)
        # tridiagonalisation route: None = automatic, True = one-stage, False = two-stage
        o.one_stage = 0 if one_stage is None else (1 if one_stage else 2)
        o.rr_one_stage = 0 if rr_one_stage is None else (1 if rr_one_stage else 2)
        self.opts = o
        h = ctypes.c_void_p()
        _check(lib().gev_setup(ctypes.byref(h), n, GEV_C128 if complex_ else GEV_F64, ctypes.byref(o)),
               "gev_setup")
        self.h = h
        self.last_report = None

    def close(self):
        if getattr(self, "h", None):
            lib().gev_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reuse_factor(self, enable: bool = True):
        _check(lib().gev_reuse_factor(self.h, 1 if enable else 0), "gev_reuse_factor")

    def _empty(self, rows, cols, dtype=None):
        import torch

        return torch.empty((cols, rows), dtype=dtype or self.dtype, device=self.device)

    # full solve on column-major buffers ------------------------------------------------------
    def solve_cm(self, Hb, Sb, k: int, evals=None, Cb=None):
        """H, S: column-major buffers (S may be None after ``reuse_factor(True)``)."""
        import torch

        n = self.n
        if evals is None:
            evals = torch.empty(k, dtype=torch.float64, device=self.device)
        if Cb is None:
            Cb = self._empty(n, k)
        rep = Report()
        code = lib().gev_solve(self.h, _ptr(Hb), n, _ptr(Sb), n, k, _ptr(evals), _ptr(Cb), n,
                               ctypes.byref(rep))
        self.last_report = rep.as_dict()
        _check(code, "gev_solve", rep.info)
        return evals, Cb

    def solve_reduced_cm(self, Hb, Sb, delta: float, k: int, evals=None, Cb=None):
        """Ill-conditioned overlap: the k lowest pairs in the eigenbasis of S with eigenvalues >= delta
        (S may be None after ``reuse_factor(True)``).  Returns (evals, C, m) with m the kept basis size."""
        import torch

        n = self.n
        if evals is None:
            evals = torch.empty(k, dtype=torch.float64, device=self.device)
        if Cb is None:
            Cb = self._empty(n, k)
        rep = Report()
        m = ctypes.c_int(0)
        code = lib().gev_solve_reduced(self.h, _ptr(Hb), n, _ptr(Sb), n, float(delta), k, _ptr(evals), _ptr(Cb), n,
                                       ctypes.byref(m), ctypes.byref(rep))
        self.last_report = rep.as_dict()
        self.last_report["m_kept"] = m.value
        _check(code, "gev_solve_reduced", m.value if code == 9 else 0)
        return evals, Cb, m.value

    def solve(self, H, S, k: int):
        """Logical torch matrices (n x n) in, (eigenvalues[k], C[n x k]) out."""
        Hb = cm(H.to(self.device, self.dtype))
        Sb = cm(S.to(self.device, self.dtype)) if S is not None else None
        w, Cb = self.solve_cm(Hb, Sb, k)
        return w, logical(Cb)

    def density(self, Cb, occ, evals=None, P=None, PE=None):
        """Density matrix P_ij = sum_l f_l conj(C_il) C_jl of the columns of C (column-major buffer,
        n x k) with occupations ``occ`` (device, k doubles); with ``evals`` also the energy-weighted
        PE (weights f_l lambda_l).  Returns P, or (P, PE): column-major n x n buffers."""
        import torch

        n = self.n
        k = Cb.shape[0]
        if Cb.shape[1] != n or not Cb.is_contiguous():
            raise ValueError("C must be a contiguous column-major n x k buffer")
        if P is None:
            P = self._empty(n, n)
        if evals is not None and PE is None:
            PE = self._empty(n, n)
        occ = occ.to(self.device, torch.float64).contiguous()
        ev = evals.to(self.device, torch.float64).contiguous() if evals is not None else None
        if occ.numel() < k or (ev is not None and ev.numel() < k):
            raise ValueError("occ and evals need k entries")
        for M in (P, PE):
            if M is not None and (tuple(M.shape) != (n, n) or not M.is_contiguous() or M.dtype != self.dtype):
                raise ValueError("P and PE must be contiguous n x n buffers of the handle's dtype")
        _check(lib().gev_density(self.h, k, _ptr(Cb), n, _ptr(occ), _ptr(ev), _ptr(P), n, _ptr(PE), n),
               "gev_density")
        return P if evals is None else (P, PE)

    def check(self, Hb, Sb, evals, Cb):
        """(resid, ortho) of the eigenpairs (evals, C) of the pencil (H, S), measured on the device:
        ||HC - SC Lambda||_1/(||H||_1 ||C||_1) and ||C^H S C - I||_1 (column-major buffers)."""
        n = self.n
        k = Cb.shape[0]
        r = ctypes.c_double(0.0)
        o = ctypes.c_double(0.0)
        _check(lib().gev_check(self.h, _ptr(Hb), n, _ptr(Sb), n, k, _ptr(evals), _ptr(Cb), n,
                               ctypes.byref(r), ctypes.byref(o)), "gev_check")
        return r.value, o.value

    # individual steps (include/gev_steps.h) --------------------------------------------------
    def potrf(self, Ab):
        info = ctypes.c_int(0)
        code = lib().gev_step_potrf(self.h, _ptr(Ab), self.n, ctypes.byref(info))
        if code not in (0, 1):
            _check(code, "gev_step_potrf")
        return info.value

    def trtri(self, Ab):
        _check(lib().gev_step_trtri(self.h, _ptr(Ab), self.n), "gev_step_trtri")

    def hegst(self, Hb, Xb, Ab=None):
        if Ab is None:
            Ab = self._empty(self.n, self.n)
        _check(lib().gev_step_hegst(self.h, _ptr(Hb), self.n, _ptr(Xb), self.n, _ptr(Ab), self.n),
               "gev_step_hegst")
        return Ab

    def he2hb(self, Ab, b: int = 0) -> int:
        used = ctypes.c_int(0)
        _check(lib().gev_step_he2hb(self.h, _ptr(Ab), self.n, b, ctypes.byref(used)), "gev_step_he2hb")
        return used.value

    def he2td(self, Ab):
        """One-stage tridiagonalisation of the Hermitian Ab (column-major, overwritten): (d, e)."""
        import torch

        d = torch.empty(self.n, dtype=torch.float64, device=self.device)
        e = torch.empty(max(self.n - 1, 1), dtype=torch.float64, device=self.device)
        _check(lib().gev_step_he2td(self.h, _ptr(Ab), self.n, _ptr(d), _ptr(e)), "gev_step_he2td")
        return d, e[: self.n - 1]

    def hb2st(self):
        import torch

        d = torch.empty(self.n, dtype=torch.float64, device=self.device)
        e = torch.empty(max(self.n - 1, 1), dtype=torch.float64, device=self.device)
        _check(lib().gev_step_hb2st(self.h, _ptr(d), _ptr(e)), "gev_step_hb2st")
        return d, e[: self.n - 1]

    def stedc(self, d, e, k: int):
        import torch

        n = self.n
        w = torch.empty(n, dtype=torch.float64, device=self.device)
        Zb = self._empty(n, k, torch.float64)
        ee = e if e.numel() > 0 else torch.zeros(1, dtype=torch.float64, device=self.device)
        defl = ctypes.c_int(0)
        _check(lib().gev_step_stedc(self.h, _ptr(d), _ptr(ee), k, _ptr(w), _ptr(Zb), n,
                                    ctypes.byref(defl)), "gev_step_stedc")
        return w, Zb, defl.value

    def back(self, Zb, k: int):
        Yb = self._empty(self.n, k)
        _check(lib().gev_step_back(self.h, _ptr(Zb), self.n, k, _ptr(Yb), self.n), "gev_step_back")
        return Yb

    def mult(self, Xb, Yb, k: int):
        Cb = self._empty(self.n, k)
        _check(lib().gev_step_mult(self.h, _ptr(Xb), self.n, _ptr(Yb), self.n, k, _ptr(Cb), self.n),
               "gev_step_mult")
        return Cb


def solve(H, S, k: int, **kw):
    """One-shot generalized solve: the k lowest eigenpairs of the pencil (H, S) (torch, on GPU)."""
    with Solver(H.shape[0], complex_=H.is_complex(), device=H.device, **kw) as s:
        return s.solve(H, S, k)
