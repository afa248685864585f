"""The C-ABI library builds for sm_103a, loads, and exports every entry point declared in
include/*.h; argument checks that need no GPU return the documented codes."""
import ctypes
import glob
import os
import re

import pytest

from paper_2502_02460_gb300 import build, gev

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return gev.lib()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(gev_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(L, nm), nm
    assert set(gev.SYMBOLS) <= set(names)


def test_workspace_and_strerror_need_no_gpu(L):
    o = gev.Opts()
    L.gev_default_opts(ctypes.byref(o))
    assert o.refine_max_iter == 4 and abs(o.refine_tol - 1e-11) < 1e-20
    b1 = L.gev_workspace_bytes(1024, 0, ctypes.byref(o))
    b2 = L.gev_workspace_bytes(1024, 1, ctypes.byref(o))
    assert b1 > 8 * 1024 * 1024 * 8 and b2 > b1
    assert L.gev_workspace_bytes(0, 0, None) == 0
    assert L.gev_workspace_bytes(10, 7, None) == 0
    assert L.gev_strerror(1) == b"S is not positive definite"
    assert L.gev_strerror(-3) == b"invalid argument"


def test_invalid_arguments_rejected_before_device_use(L):
    h = ctypes.c_void_p()
    assert L.gev_setup(None, 10, 0, None) == -1
    assert L.gev_setup(ctypes.byref(h), 0, 0, None) == -2
    assert L.gev_setup(ctypes.byref(h), 10, 5, None) == -3
    assert L.gev_solve(None, None, 1, None, 1, 1, None, None, 1, None) == -1
    assert L.gev_free(None) == 0
    assert L.gev_reuse_factor(None, 1) == -1
    for fn, nargs in (("gev_step_potrf", 4), ("gev_step_trtri", 3), ("gev_step_hegst", 7),
                      ("gev_step_he2hb", 5), ("gev_step_hb2st", 3), ("gev_step_stedc", 8),
                      ("gev_step_back", 6), ("gev_step_mult", 8)):
        f = getattr(L, fn)
        args = [None] + [None if t in (ctypes.c_void_p,) or hasattr(t, "contents") else 0
                         for t in f.argtypes[1:]]
        assert f(*args) == -1, fn


def test_oracle_is_not_imported_by_the_package():
    pkg = os.path.join(ROOT, "paper_2502_02460_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            txt = open(f).read()
            assert "import oracle" not in txt and "oracle_gev" not in txt and "from oracle" not in txt, f


def test_emulated_gemm_scratch_size_needs_no_gpu(L):
    """The digit planes take 16 bytes per padded element of op(A) and op(B) (8 BF16 planes), with K
    capped at one launch's 32768; negative sizes give 0."""
    f = L.gev_gemm_f64_scratch_bytes
    f.argtypes = [ctypes.c_int] * 3
    f.restype = ctypes.c_size_t
    assert f(-1, 5, 5) == 0
    b = f(1000, 500, 3000)
    assert b >= 16 * (1024 + 512) * 3008
    assert f(1000, 500, 40000) == f(1000, 500, 32768)
    assert f(10, 10, 0) > 0


def test_fp32_tensor_gemm_scratch_size_needs_no_gpu(L):
    """Three BF16 planes (6 bytes) per padded element of op(A) (rows to 128) and op(B) (columns to 256)."""
    f = L.gev_gemm_f32_scratch_bytes
    f.argtypes = [ctypes.c_int] * 3
    f.restype = ctypes.c_size_t
    assert f(5, -1, 5) == 0
    assert f(1000, 500, 3000) >= 6 * (1024 + 512) * 3008
    assert f(0, 0, 0) > 0
