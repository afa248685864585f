"""Time the matrix-product entry points of include/gev_kernels.h on one GPU.

    python -m paper_2502_02460_gb300.gemm_bench --dtype f64 --engine 1 --m 8192 --n 8192 --k 8192

f64 engine 1: FP64 product emulated on the BF16 tensor cores (digit planes); f64 engine 0: native
FP64 DMMA; f32 engines 1 / 2: BF16x6 / BF16x3 split products on the tensor cores; f32 engine 0:
FP32 CUDA-core FMAs.  Prints
one JSON line: milliseconds per call (CUDA events around the C-ABI call, which synchronises), the
algorithmic TFLOP/s (2 M N K per call), and the largest error against torch's product of the same
operands relative to (|A| |B|)_ij.
"""
from __future__ import annotations

import argparse
import ctypes
import json

from . import gev


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    ap.add_argument("--engine", type=int, choices=[0, 1, 2], default=1)
    ap.add_argument("--m", type=int, default=4096)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--k", type=int, default=4096)
    ap.add_argument("--ta", type=int, choices=[0, 1], default=0)
    ap.add_argument("--tb", type=int, choices=[0, 1], default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--beta", type=float, default=0.0, help="C = op(A) op(B) + beta C (C starts random)")
    args = ap.parse_args(argv)

    import torch

    L = gev.lib()
    vp, i = ctypes.c_void_p, ctypes.c_int
    dev = torch.device("cuda:0")
    M, N, K = args.m, args.n, args.k
    dt = torch.float64 if args.dtype == "f64" else torch.float32
    g = torch.Generator(device=dev).manual_seed(args.seed)
    # stored matrices, column-major (a row-major (cols x rows) tensor)
    a_rows, a_cols = (M, K) if args.ta == 0 else (K, M)
    b_rows, b_cols = (K, N) if args.tb == 0 else (N, K)
    A = torch.randn(a_cols, a_rows, generator=g, device=dev, dtype=dt)
    B = torch.randn(b_cols, b_rows, generator=g, device=dev, dtype=dt)
    C0 = torch.randn(N, M, generator=g, device=dev, dtype=dt)
    C = C0.clone()
    st = torch.zeros(16, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    if args.dtype == "f64":
        L.gev_gemm_f64.argtypes = [i, i, i, i, i, ctypes.c_double, vp, i, vp, i, ctypes.c_double, vp, i, i, vp,
                                   vp, vp, ctypes.c_size_t]
        L.gev_gemm_f64.restype = i
        L.gev_gemm_f64_scratch_bytes.argtypes = [i, i, i]
        L.gev_gemm_f64_scratch_bytes.restype = ctypes.c_size_t
        nbytes = L.gev_gemm_f64_scratch_bytes(M, N, K) if args.engine == 1 else 0
        scr = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)

        def call():
            return L.gev_gemm_f64(M, N, K, args.ta, args.tb, 1.0, vp(A.data_ptr()), a_rows, vp(B.data_ptr()), b_rows,
                                  args.beta, vp(C.data_ptr()), M, args.engine, vp(stream.cuda_stream),
                                  vp(st.data_ptr()), vp(scr.data_ptr()), nbytes)
    else:
        L.gev_gemm_f32.argtypes = [i, i, i, i, i, ctypes.c_float, vp, i, vp, i, ctypes.c_float, vp, i, i, vp, vp,
                                   vp, ctypes.c_size_t]
        L.gev_gemm_f32.restype = i
        L.gev_gemm_f32_scratch_bytes.argtypes = [i, i, i]
        L.gev_gemm_f32_scratch_bytes.restype = ctypes.c_size_t
        nbytes = L.gev_gemm_f32_scratch_bytes(M, N, K) if args.engine > 0 else 0
        scr = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)

        def call():
            return L.gev_gemm_f32(M, N, K, args.ta, args.tb, 1.0, vp(A.data_ptr()), a_rows, vp(B.data_ptr()), b_rows,
                                  args.beta, vp(C.data_ptr()), M, args.engine, vp(stream.cuda_stream),
                                  vp(st.data_ptr()), vp(scr.data_ptr()), nbytes)

    for _ in range(args.warmup):
        C.copy_(C0)
        if call() != 0:
            raise gev.GevError(-1, "gemm call")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.reps):
        if call() != 0:
            raise gev.GevError(-1, "gemm call")
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.reps, 1)
    C.copy_(C0)  # one more call from the initial C for the error check
    if call() != 0:
        raise gev.GevError(-1, "gemm call")
    torch.cuda.synchronize()
    if int(st[1].item()) != 0:
        raise gev.GevError(3, "gemm call (bounded wait expired)")
    opA = A.T if args.ta == 0 else A  # (M x K) logical
    opB = B.T if args.tb == 0 else B
    ref = opA.double() @ opB.double() + args.beta * C0.T.double()
    scale = opA.double().abs() @ opB.double().abs() + abs(args.beta) * C0.T.double().abs()
    err = ((C.T.double() - ref).abs() / scale.clamp_min(1e-300)).max().item()
    print(json.dumps({"dtype": args.dtype, "engine": args.engine, "m": M, "n": N, "k": K, "ta": args.ta,
                      "tb": args.tb, "beta": args.beta, "ms_per_call": ms, "tflops": 2.0 * M * N * K / (ms * 1e-3) / 1e12,
                      "max_rel_err": err, "status": int(st[1].item())}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
