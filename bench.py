"""Benchmark: time-to-solution of the dense generalized Hermitian eigensolve H C = S C Lambda.

Workload (default): the N=16384 real configuration (k = 4096 lowest eigenpairs, seed 3, Toeplitz
overlap and DFT-like spectrum; see paper_2502_02460_gb300/inputs.py).  A step is one complete
gev_solve (Cholesky, inversion, Multiply, full->band, bulge chasing, divide and conquer, both
back-transforms, C = X^H Y) on inputs already resident in HBM.  H and S are 2 x 2.1 GB, far larger
than L2 (129 MB), so no L2 flush is needed between steps.

Printed (rank 0, one JSON line): seconds per solve (lower is better), the roofline entry of the
FP64 matrix products (algorithmic flops of every launch / CUDA-event time of every launch, on the
solve stream; for products emulated on the BF16 tensor cores, 36 digit-pair products each against
the BF16 peak), the plain FP64 form beside the mixed headline (native and emulated products), the
CPU oracle on a bounded sample, the end-to-end time through the Python API with pinned host
buffers, the number of kernels launched, SM clocks sampled during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--n N --k K] [--impl reference]

Multi-GPU (torchrun, one rank per GPU): every rank solves its own independent system (k-points /
spin channels are independent problems), no collective on the data path; value = solves of all
ranks / max-over-ranks time ("weak" scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "N=16384 gen. eigensolve s (FP64 vs mixed, resid≤1e-11); k-pt stream p50/p99 ms"
FP64_NOMINAL_TF = 1.25      # GB300 FP64 (DMMA) nominal, dense
BF16_NOMINAL_TF = 2250.0    # GB300 BF16 nominal, dense
EMU_PAIRS = 36              # BF16 digit-pair products per emulated FP64 product (p + q <= 9, 8 planes)
# DRAM bytes of one ozaki_kernel launch, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum,
# --clock-control none) of the 4096^3 product, the order of the solve's largest products; the timed
# products of a solve differ in shape, so the figure is that launch's, not a per-solve average
OZAKI_TRAFFIC = {"bytes": 2.579e9 + 0.132e9,
                 "case": "ozaki_kernel, one 4096x4096x4096 FP64 product (profiles/ozaki_kernel_gemm_f64_4096.md)"}
FP64_FMA_TF = 1.00          # GB300 FP64 FMA pipe of the CUDA cores, measured (probe kernel)
FP32_FMA_TF = 73.9          # GB300 FP32 FMA pipe of the CUDA cores, measured (probe kernel)


def steps_roofline(step_ms, n, k, b, complex_, mixed, emulated, refine_iters, fp32_products, mp):
    """Per-step rates: each step's algorithmic flops (real counts, x4 for complex data) over its
    measured CUDA-event time, against the peak of the engine that runs the step's arithmetic.

    Peaks: FP64 products emulated on the BF16 tensor cores count 36 BF16 digit-pair products per FP64
    product (FP64-equivalent peak = BF16 sustained / 36); FP32 products as BF16x6 (x3) split products
    count 6 (3) BF16 products; native FP64 products run at the BF16 sustained rate times the nominal
    FP64/BF16 ratio; element-wise FMA work on the CUDA cores uses the measured FMA-pipe rates.  The
    divide-and-conquer step has no fixed flop count (deflation decides it) and reports its time only;
    the refinement counts its FP64 work only."""
    F = 4.0 if complex_ else 1.0
    N, K, B = float(n), float(k), float(b)
    bf16 = float(mp.get("bf16_tflops_sustained", 1764.7))
    if emulated:
        fp64 = ("FP64 products emulated on BF16 tcgen05 (36 digit-pair MMAs each)", bf16 / EMU_PAIRS)
    else:
        fp64 = ("FP64 products on DMMA (mma.sync m8n8k4)", bf16 * FP64_NOMINAL_TF / BF16_NOMINAL_TF)
    if fp32_products == 0:
        fp32 = ("FP32 products on the CUDA cores", FP32_FMA_TF)
    elif fp32_products == 3:
        fp32 = ("FP32 products as BF16x3 on tcgen05 (thin ones on the CUDA cores)", bf16 / 3)
    else:
        fp32 = ("FP32 products as BF16x6 on tcgen05 (thin ones on the CUDA cores)", bf16 / 6)
    low_real = mixed and not complex_
    if not mixed:
        fma = ("FP64 FMA on the CUDA cores", FP64_FMA_TF)
    else:
        fma = ("FP32 (complex64) FMA on the CUDA cores", FP32_FMA_TF)
    # back-transform 2: compact-WY tensor-core products on the emulated engine, else reflector by
    # reflector on the FMA pipe; the mixed form back-transforms all N FP32 vectors (the refinement
    # uses the complement), the plain forms the k wanted ones
    bt2 = fp64 if (emulated and not mixed) else fma
    KB = N if mixed else K
    work = {
        "cholesky": (2.0 * N ** 3 / 3.0, fp64),  # Cholesky and inversion, one fused recursion
        "multiply": (N ** 3, fp64),
        "to_band": (4.0 * N ** 3 / 3.0, fp32 if low_real else fp64),
        "to_tridiag": (6.0 * B * N * N, fma),  # bulge chasing: bound by the 3N-task critical path
        "solve": (None, ("secular equations in FP64 on the CUDA cores; merge products on the product engine",
                         None)),
        "back_tridiag": (2.0 * N * N * KB, bt2),
        "back_band": (2.0 * N * N * KB, fp32 if low_real else fp64),
        "mult": (N * N * K, fp64),
    }
    if mixed:
        work["refine"] = (refine_iters * (2.0 * N * N * K + 3.0 * N * K * K), fp64)
    out = {}
    for step, (flops, (engine, peak)) in work.items():
        ms = float(step_ms.get(step, 0.0) or 0.0)
        row = {"ms": ms, "engine": engine}
        if flops is not None and ms > 0:
            tf = F * flops / (ms * 1e-3) / 1e12
            row.update({"flops": F * flops, "tflops": tf, "peak_tflops": peak,
                        "frac": tf / peak if peak else None})
        out[step] = row
    return out


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            mp = json.load(f)
        return mp, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(os.environ.get("GEV_BENCH_OUT", tempfile.gettempdir()), f"gev_clocks_rank{index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model() -> str:
    """Host CPU description for the baseline record: the kernel's model name, else the architecture
    with its CPU part / implementer codes."""
    import platform

    name, part, impl = None, None, None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key, _, val = line.partition(":")
                key, val = key.strip(), val.strip()
                if key == "model name" and not name:
                    name = val
                elif key == "CPU part" and not part:
                    part = val
                elif key == "CPU implementer" and not impl:
                    impl = val
    except OSError:
        pass
    if name:
        return name
    return f"{platform.machine()} (implementer {impl}, part {part})" if part else platform.machine()


def cpu_baseline(n_full: int, k_full: int, complex_: bool, seconds_target: float = 15.0):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the same recipe, scaled to the
    metric's unit (seconds per N=n_full solve) by the cubic cost of the dense solve."""
    import numpy as np

    import oracle
    from paper_2502_02460_gb300 import inputs

    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    ns = 512
    t = 0.0
    while True:
        p = inputs.make_problem(ns, max(1, ns * k_full // n_full), seed=3, complex_=complex_)
        t0 = time.perf_counter()
        w, C, info, dg = oracle.gev(p.H, p.S, max(1, ns * k_full // n_full))
        t = time.perf_counter() - t0
        if t >= seconds_target / 8 or ns >= 2048:
            break
        ns *= 2
    scaled = t * (n_full / ns) ** 3
    return {"value": scaled, "unit": "s", "cores": int(os.environ.get("OMP_NUM_THREADS", cores)),
            "kind": "oracle", "cpu": cpu_model(),
            "sample": f"oracle on N={ns}, k={max(1, ns * k_full // n_full)} of the same recipe "
                      f"({t:.2f} s), scaled by (N/{ns})^3 to N={n_full}"}


def oracle_full_configs(threads_list=(None, 1), include_n4096=True):
    """The FP64 CPU oracle, as it stands, timed IN FULL (no sampling, no scaling) on the two
    configurations small enough for it: real N=512 with all 512 eigenpairs (seed 0) and real N=4096
    with the k=1229 lowest (seed 1, 1e-8 cluster of 16).  N=512 runs at every thread count in
    ``threads_list`` (None = all host cores); N=4096 at all host cores only (about a minute; a
    single core would take about 20)."""
    import numpy as np

    import oracle
    from paper_2502_02460_gb300 import inputs

    oracle.lib()
    cores = os.cpu_count() or 1
    try:
        import ctypes
        omp = ctypes.CDLL("libgomp.so.1")
        set_threads = omp.omp_set_num_threads
        set_threads.argtypes = [ctypes.c_int]
    except OSError:
        set_threads = None
    out = []
    cases = [(512, 512, 0, False)] + ([(4096, 1229, 1, True)] if include_n4096 else [])
    for n, k, seed, cluster in cases:
        p = inputs.make_problem(n, k, seed=seed, cluster=cluster)
        for th in (threads_list if n <= 512 else (None,)):
            nt = cores if th is None else th
            if set_threads is not None:
                set_threads(nt)
            t0 = time.perf_counter()
            w, C, info, dg = oracle.gev(p.H, p.S, k)
            t = time.perf_counter() - t0
            out.append({"n": n, "k": k, "seed": seed, "threads": nt if set_threads else None, "s": t,
                        "info": info, "max_abs_eig_err_vs_construction": float(np.max(np.abs(w - p.lam[:k]))),
                        "resid": dg["resid"], "ortho": dg["ortho"]})
        try:  # context only: LAPACK through scipy on the same cores (neither the oracle nor the target)
            import scipy.linalg as sla

            t0 = time.perf_counter()
            ws = sla.eigh(p.H, p.S, subset_by_index=[0, k - 1], eigvals_only=False)[0]
            out.append({"n": n, "k": k, "context": "scipy.linalg.eigh (LAPACK)", "s": time.perf_counter() - t0,
                        "max_abs_eig_err_vs_construction": float(np.max(np.abs(ws - p.lam[:k])))})
        except ImportError:
            pass
    if set_threads is not None:
        set_threads(cores)
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    vals = []
    sample = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(args.n, args.k, args.complex, seconds_target=4.0)
        if i >= args.warmup:
            vals.append(cb["value"])
        sample = cb["sample"]
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "cpu": cpu_model(), "sample": sample, "value": v,
                             "unit": "s"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_stream(args, dev, mixed=False):
    """A prefix of the k-point serving stream (Poisson arrivals at 200/s, complex128 pencils of
    log-uniform size recurring for 10 SCF iterations with fixed S, k = N/4) through the
    continuous-batching server; latency from each request's scheduled arrival to its result."""
    import numpy as np
    import torch

    from paper_2502_02460_gb300 import gev, inputs, serve

    spec = serve.StreamSpec(requests=args.stream_requests, n_max=args.stream_n_max)
    plan = serve.stream_plan(spec)
    cache = {}
    for (_, sid, it, n, k, last) in plan:  # build every request's pencil before the clock starts
        on_gpu = n > 2048  # the construction's dense algebra through torch on the device (input only)
        if sid not in cache:
            p = inputs.make_problem(n, k, seed=4000 + sid, complex_=True, gap_check=False,
                                    device=dev if on_gpu else None)
            cache[sid] = (p, p.S if on_gpu else gev.cm_from_numpy(p.S, dev))
        p = cache[sid][0]
        if on_gpu:  # p.H: column-major device buffer (the row-major buffer of H^T)
            H0 = p.H
            if it == 0:
                cache[(sid, it)] = H0
                continue
            rng = np.random.default_rng(5000 + 1000 * sid + it)
            G = torch.from_numpy(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).to(dev)
            dH = 0.5 * (G + G.conj().transpose(0, 1))
            del G
            dH = dH.transpose(0, 1).contiguous()  # column-major buffer of the Hermitian dH
            scale = spec.dh_rel * torch.linalg.norm(H0) / torch.linalg.norm(dH)
            cache[(sid, it)] = H0 + scale * dH
            del dH
            continue
        rng = np.random.default_rng(5000 + 1000 * sid + it)
        G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        dH = 0.5 * (G + G.conj().T)
        H = p.H + (spec.dh_rel * np.linalg.norm(p.H) / np.linalg.norm(dH) * dH if it > 0 else 0)
        cache[(sid, it)] = gev.cm_from_numpy(H, dev)
    torch.cuda.synchronize()
    srv = serve.Server(budget_bytes=120e9, workers=args.stream_workers, device=dev, mixed=mixed)
    t0 = time.perf_counter()
    futs = []
    for (t, sid, it, n, k, last) in plan:
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        futs.append(srv.submit(sid, cache[(sid, it)], cache[sid][1] if it == 0 else None, k, n=n,
                               complex_=True, last=last, arrival=t0 + t))
    for f in futs:
        f.result()
    srv.close()
    st = srv.stats()
    st.update({"precision": "mixed (FP32 band reduction + FP64 refinement)" if mixed else "plain FP64",
               "dtype": "c128",
               "workers": args.stream_workers,
               "workload": f"first {spec.requests} requests of the k-point stream (Poisson 200/s, "
                           f"N log-uniform in [{spec.n_min}, {spec.n_max}], 10 SCF iterations per "
                           f"system, S fixed, k = N/4)"})
    return st


def run_stream_only(args):
    """The k-point serving stream alone (plain FP64 and mixed), one JSON line."""
    import torch

    from paper_2502_02460_gb300 import build

    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    clocks = ClockSampler(dev.index)
    clocks.start()
    t0 = time.perf_counter()
    plain = run_stream(args, dev)
    mixed = run_stream(args, dev, mixed=True)
    clk = clocks.stop()
    print(json.dumps({"metric": "k-point stream p50/p99 ms, solves/s", "stream": plain, "stream_mixed": mixed,
                      "wall_s": time.perf_counter() - t0, "clocks": clk}), flush=True)
    return 0


CONFIGS = [  # (name, n, k, seed, complex, cluster)
    ("config 0: real N=512, all pairs, seed 0", 512, 512, 0, False, False),
    ("config 1: real N=4096, k=1229, seed 1, 1e-8 cluster of 16", 4096, 1229, 1, False, True),
    ("config 2: complex128 N=20000, k=5000, seed 2", 20000, 5000, 2, True, False),
]


def one_stage_opt(args):
    """--one-stage as the Solver's one_stage argument (None = automatic)."""
    return {"auto": None, "on": True, "off": False}[getattr(args, "one_stage", "auto")]


def run_configs(args):
    """The smaller configurations timed on the GPU (plain FP64 with emulated and native products, and
    the mixed form): median of ``--steps`` solves after ``--warmup``, CUDA events on the solve
    stream, inputs resident; eigenvalue error against the construction and the on-device
    residual / orthogonality of one more solve."""
    import numpy as np
    import torch

    from paper_2502_02460_gb300 import build, gev, inputs

    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    out = []
    for name, n, k, seed, cx, cluster in CONFIGS:
        if args.configs_max_n and n > args.configs_max_n:
            continue
        on_gpu = n > 4096
        p = inputs.make_problem(n, k, seed=seed, complex_=cx, cluster=cluster, device=dev if on_gpu else None,
                                gap_check=not on_gpu)
        Hb, Sb = (p.H, p.S) if on_gpu else (gev.cm_from_numpy(p.H, dev), gev.cm_from_numpy(p.S, dev))
        h1 = float(Hb.abs().sum(dim=1).max().item())
        rows = {}
        forms = [("plain_emulated", False, 1), ("mixed", True, -1)]
        if n <= 4096:
            forms.insert(1, ("plain_native", False, 0))
        for form, mixed, emu in forms:
            with gev.Solver(n, complex_=cx, device=dev, mixed=mixed, fp64_emulation=emu, timing=1, stream=stream,
                            check=True) as sv:
                w = torch.empty(k, dtype=torch.float64, device=dev)
                Cb = torch.empty((k, n), dtype=sv.dtype, device=dev)
                sv.solve_cm(Hb, Sb, k, w, Cb)
                acc = {"resid": sv.last_report["resid"], "ortho": sv.last_report["ortho"]}
                sv.opts.check = 0
            with gev.Solver(n, complex_=cx, device=dev, mixed=mixed, fp64_emulation=emu, timing=1,
                            stream=stream) as sv:
                for _ in range(args.warmup):
                    sv.solve_cm(Hb, Sb, k, w, Cb)
                times, steps = [], []
                for _ in range(args.steps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    sv.solve_cm(Hb, Sb, k, w, Cb)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1) / 1e3)
                    steps.append(sv.last_report["ms"])
            err = float(np.max(np.abs(w.cpu().numpy() - p.lam[:k])))
            rows[form] = {"s": statistics.median(times), "per_step_s": times,
                          "steps_ms": {kk: statistics.median(r[kk] for r in steps) for kk in gev.STEP_NAMES},
                          "max_abs_eig_err_vs_construction": err, "err_over_h1": err / h1, **acc}
        out.append({"config": name, "n": n, "k": k, "complex": cx, "h1": h1, "forms": rows,
                    "steps": args.steps, "warmup": args.warmup})
        del Hb, Sb, p
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "time-to-solution of configurations 0-2 (s)", "configs": out}), flush=True)
    return 0


def time_density(solver, Cb, w, Sb, dev, stream, reps=5, warmup=3):
    """Density matrix and energy-weighted density matrix (gev_density) of the benchmarked orbitals,
    every orbital doubly occupied; CUDA events on the solver's stream around ``reps`` calls."""
    import torch

    k, n = Cb.shape
    occ = torch.full((k,), 2.0, dtype=torch.float64, device=dev)
    P = solver._empty(n, n)
    PE = solver._empty(n, n)
    for _ in range(warmup):
        solver.density(Cb, occ, w, P=P, PE=PE)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        solver.density(Cb, occ, w, P=P, PE=PE)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # electron count: sum_ij P_ij S_ij = sum_l f_l (S-orthonormal orbitals)
    ne = float(torch.sum(P * Sb).real.item())
    flops = 2 * (n * (n + 1) // 2) * k * (8 if solver.complex else 2)  # P and PE, lower triangles
    del P, PE
    return {"ms_per_call": ms, "matrices": 2, "reps": reps, "warmup": warmup,
            "fp64_tflops": flops / (ms * 1e-3) / 1e12,
            "electron_count_rel_err": abs(ne - 2.0 * k) / (2.0 * k)}


def workload_config(args):
    return {"workload": f"{'complex128' if args.complex else 'real'} N={args.n}, k={args.k} lowest "
                        f"eigenpairs, seed {args.seed}, Toeplitz S, DFT-like spectrum; "
                        f"{'mixed' if args.mixed else 'plain FP64'} path",
            "n": args.n, "k": args.k, "precision": "mixed" if args.mixed else "plain",
            "band_b": args.band_b, "tridiag_route": getattr(args, "one_stage", "auto"),
            "l2": "inputs (2 x n^2 x 8 B) larger than L2; no flush needed"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--k", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--complex", action="store_true")
    ap.add_argument("--mixed", dest="mixed", action="store_true", default=True,
                    help="headline = mixed form (default)")
    ap.add_argument("--plain", dest="mixed", action="store_false", help="headline = plain FP64 form")
    ap.add_argument("--no-plain-beside", action="store_true",
                    help="do not time the plain FP64 solve beside the mixed headline")
    ap.add_argument("--plain-steps", type=int, default=5,
                    help="timed solves of the plain FP64 form (emulated products) beside the headline")
    ap.add_argument("--plain-native-steps", type=int, default=3,
                    help="timed solves of the plain FP64 form with native DMMA products")
    ap.add_argument("--no-oracle-configs", action="store_true",
                    help="skip timing the oracle in full on the N=512 and N=4096 configurations")
    ap.add_argument("--stream-requests", type=int, default=32,
                    help="requests of the k-point serving stream reported beside (0 = none)")
    ap.add_argument("--stream-n-max", type=int, default=2048)
    ap.add_argument("--stream-workers", type=int, default=12,
                    help="concurrent solves of the serving stream (each on its own handle and stream; the "
                         "device-memory budget of 120 GB bounds the large ones)")
    ap.add_argument("--stream-full", action="store_true",
                    help="the whole k-point stream: 512 requests, N log-uniform in [256, 8192]")
    ap.add_argument("--configs", action="store_true",
                    help="time configurations 0-2 (N=512 all pairs; N=4096 k=1229 cluster; complex N=20000 "
                         "k=5000) in every form and print one line")
    ap.add_argument("--configs-max-n", type=int, default=0, help="--configs: skip orders above this (0 = none)")
    ap.add_argument("--stream-only", action="store_true",
                    help="run only the k-point stream (both precisions) and print its line")
    ap.add_argument("--band-b", type=int, default=64)
    ap.add_argument("--one-stage", default="auto", choices=["auto", "on", "off"],
                    help="tridiagonalisation route of the headline solve (gev_opts.one_stage)")
    ap.add_argument("--fp32-products", type=int, default=-1, choices=[-1, 0, 3, 6],
                    help="mixed form, FP32 products: 6 / 3 = BF16x6 / BF16x3 on the tensor cores, "
                         "0 = FP32 CUDA cores, -1 = automatic")
    ap.add_argument("--rr-band-b", type=int, default=0, choices=[0, 16, 32, 64],
                    help="mixed form: band width of the refinement's Rayleigh-Ritz solve (0 = automatic)")
    ap.add_argument("--fp64-emulation", type=int, default=-1, choices=[-1, 0, 1],
                    help="FP64 products of the headline solve: 1 = BF16 digit planes on the tensor "
                         "cores, 0 = native DMMA, -1 = automatic (1)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-check", action="store_true",
                    help="skip the on-device accuracy measurement of one extra solve")
    ap.add_argument("--no-density", action="store_true",
                    help="skip timing the density-matrix output of the benchmarked orbitals")
    ap.add_argument("--gen", default="auto", choices=["auto", "cpu", "gpu"],
                    help="where the synthetic pencil is built (auto: GPU for N > 4096)")
    args = ap.parse_args()
    if args.stream_full:
        args.stream_requests, args.stream_n_max = 512, 8192
    if args.impl == "reference":
        return run_reference(args)
    if args.stream_only:
        return run_stream_only(args)
    if args.configs:
        return run_configs(args)

    import torch

    from paper_2502_02460_gb300 import build, gev, inputs

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    # independent system per rank (weak scaling): seed offset by rank
    on_gpu = args.gen == "gpu" or (args.gen == "auto" and args.n > 4096)
    p = inputs.make_problem(args.n, args.k, seed=args.seed + 100 * rank, complex_=args.complex,
                            device=dev if on_gpu else None, gap_check=False)
    if on_gpu:
        Hb, Sb = p.H, p.S  # column-major device buffers
    else:
        Hb, Sb = gev.cm_from_numpy(p.H, dev), gev.cm_from_numpy(p.S, dev)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    solver = gev.Solver(args.n, complex_=args.complex, device=dev, mixed=args.mixed,
                        band_b=args.band_b, timing=2, stream=stream, fp64_emulation=args.fp64_emulation,
                        fp32_products=args.fp32_products, rr_band_b=args.rr_band_b,
                        one_stage=one_stage_opt(args))
    w = torch.empty(args.k, dtype=torch.float64, device=dev)
    Cb = torch.empty((args.k, args.n), dtype=solver.dtype, device=dev)
    for _ in range(args.warmup):
        solver.solve_cm(Hb, Sb, args.k, w, Cb)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(dev.index)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    reps = []
    e0.record(stream)
    for _ in range(args.steps):
        solver.solve_cm(Hb, Sb, args.k, w, Cb)
        reps.append(solver.last_report)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    # accuracy of the benchmarked result against the construction (exact eigenvalues)
    wl = w.cpu().numpy()
    import numpy as np

    err = float(np.max(np.abs(wl - p.lam[: args.k])))
    # roofline of the dominant kernel: FP64 DMMA GEMM
    gemm_ms = sum(r["gemm_ms"] for r in reps)
    gemm_fl = sum(r["gemm_flops"] for r in reps)
    gemm_calls = sum(r["gemm_calls"] for r in reps)
    mp, src = peaks()
    emu_used = args.fp64_emulation != 0
    fp64_tf = gemm_fl / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else None
    if emu_used:
        # each FP64 product runs as 36 BF16 digit-pair products on the tensor cores
        peak = mp.get("bf16_tflops_sustained", 1764.7)
        achieved = EMU_PAIRS * fp64_tf if fp64_tf else None
        roof_kernel = ("ozaki_kernel + k_split/k_vec_exp (FP64 products as 36 BF16 digit-pair tcgen05 MMAs, "
                       "achieved = 36 x FP64 algorithmic flops / time of every FP64 product launch)")
        peak_source = f"{src} bf16_tflops_sustained"
    else:
        peak = mp.get("bf16_tflops_sustained", 1764.7) * FP64_NOMINAL_TF / BF16_NOMINAL_TF
        achieved = fp64_tf
        roof_kernel = "gemm_kernel<double> (FP64 DMMA mma.sync m8n8k4)"
        peak_source = (f"{src} bf16 sustained x FP64/BF16 nominal ratio ({FP64_NOMINAL_TF}/{BF16_NOMINAL_TF})")
    step_ms = {k: statistics.median(r["ms"][k] for r in reps) for k in gev.STEP_NAMES}
    launches = int(statistics.median(r["launches"] for r in reps))
    # the plain FP64 form on the same input, beside the mixed headline (1 warm-up, 1 timed solve):
    # with native FP64 products (DMMA) and with FP64 products emulated on the BF16 tensor cores
    plain = plain_emu = None
    if args.mixed and not args.no_plain_beside:
        solver.close()

        def time_plain(emu, steps):
            ps = gev.Solver(args.n, complex_=args.complex, device=dev, mixed=False, band_b=args.band_b,
                            timing=1, stream=stream, fp64_emulation=emu)
            ps.solve_cm(Hb, Sb, args.k, w, Cb)
            torch.cuda.synchronize()
            times, steps_ms = [], []
            for _ in range(steps):
                f0 = torch.cuda.Event(enable_timing=True)
                f1 = torch.cuda.Event(enable_timing=True)
                f0.record(stream)
                ps.solve_cm(Hb, Sb, args.k, w, Cb)
                f1.record(stream)
                torch.cuda.synchronize()
                times.append(f0.elapsed_time(f1) / 1e3)
                steps_ms.append(ps.last_report["ms"])
            med_steps = {kk: statistics.median(r[kk] for r in steps_ms) for kk in gev.STEP_NAMES}
            out = {"value": statistics.median(times), "unit": "s", "steps": steps, "warmup": 1,
                   "per_step_s": times,
                   "fp64_products": "emulated (BF16 digit planes, tcgen05)" if emu else "native (DMMA)",
                   "steps_ms": med_steps,
                   "steps_roofline": steps_roofline(med_steps, args.n, args.k, args.band_b, args.complex,
                                                    False, emu != 0, 0, args.fp32_products, mp),
                   "max_abs_eig_err_vs_construction": float(np.max(np.abs(w.cpu().numpy() - p.lam[: args.k])))}
            ps.close()
            return out

        plain = time_plain(0, args.plain_native_steps)
        if not args.complex:
            plain_emu = time_plain(1, args.plain_steps)
        solver = gev.Solver(args.n, complex_=args.complex, device=dev, mixed=args.mixed,
                            band_b=args.band_b, timing=0, stream=stream, fp64_emulation=args.fp64_emulation,
                            fp32_products=args.fp32_products, rr_band_b=args.rr_band_b,
                        one_stage=one_stage_opt(args))
    # end-to-end through the Python API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        Hh = Hb.cpu().pin_memory()
        Sh = Sb.cpu().pin_memory()
        wh = torch.empty(args.k, dtype=torch.float64).pin_memory()
        Ch = torch.empty((args.k, args.n), dtype=solver.dtype).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Hd = Hh.to(dev, non_blocking=True)
        Sd = Sh.to(dev, non_blocking=True)
        wd, Cd = solver.solve_cm(Hd, Sd, args.k)
        wh.copy_(wd, non_blocking=True)
        Ch.copy_(Cd, non_blocking=True)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        es = 16 if args.complex else 8
        e2e = {"value": t_e2e, "unit": "s", "h2d_bytes_per_step": 2 * args.n * args.n * es,
               "d2h_bytes_per_step": args.k * 8 + args.n * args.k * es}
        del Hd, Sd
    dens = None if args.no_density else time_density(solver, Cb, w, Sb, dev, stream)
    # accuracy of the benchmarked configuration, measured on the device (gev_opts.check): the residual
    # ||HC - SC Lambda||_1/(||H||_1 ||C||_1) and ||C^H S C - I||_1 of one more solve (not timed)
    accuracy = None
    if not args.no_check:
        solver.close()
        cs = gev.Solver(args.n, complex_=args.complex, device=dev, mixed=args.mixed, band_b=args.band_b,
                        stream=stream, fp64_emulation=args.fp64_emulation, fp32_products=args.fp32_products,
                        check=True, rr_band_b=args.rr_band_b, one_stage=one_stage_opt(args))
        cs.solve_cm(Hb, Sb, args.k, w, Cb)
        accuracy = {"resid": cs.last_report["resid"], "ortho": cs.last_report["ortho"],
                    "bound_resid": 1e-11 if args.mixed else 1e-13 * args.n ** 0.5,
                    "bound_ortho": 1e-12 * args.n ** 0.5, "measured": "on the device (gev_opts.check)"}
        cs.close()
    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
        return 0
    cb = None if args.no_cpu_baseline else cpu_baseline(args.n, args.k, args.complex)
    if cb is not None and not args.no_oracle_configs:
        cb["full_size_runs"] = oracle_full_configs()
    stream_stats = stream_mixed = None
    if args.stream_requests > 0 and ws == 1:
        del solver, Hb, Sb
        torch.cuda.empty_cache()
        stream_stats = run_stream(args, dev)
        stream_mixed = run_stream(args, dev, mixed=True)
    value = ms / 1e3 / (1 if ws == 1 else 1)  # seconds per solve (each rank solves one system)
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args),
        "solves_per_s": ws / (ms / 1e3),
        "max_abs_eig_err_vs_construction": err,
        "steps_ms": step_ms,
        "steps_roofline": steps_roofline(step_ms, args.n, args.k, args.band_b, args.complex, args.mixed, emu_used,
                                         reps[-1]["refine_iters"] if args.mixed else 0, args.fp32_products, mp),
        "fp64_plain": plain,
        "fp64_plain_emulated_products": plain_emu,
        "refine": {"iterations": reps[-1]["refine_iters"], "residual": reps[-1]["refine_resid"]}
        if args.mixed else None,
        "stream": stream_stats,
        "stream_mixed": stream_mixed,
        "density": dens,
        "accuracy": accuracy,
        "roofline": {"bound": "tensor", "kernel": roof_kernel,
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": OZAKI_TRAFFIC["bytes"],
                     "traffic_case": OZAKI_TRAFFIC["case"],
                     "launches_timed": gemm_calls, "fp64_equivalent_tflops": fp64_tf,
                     "peak_source": peak_source},
        "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches * args.steps, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
    return 0


if __name__ == "__main__":
    sys.exit(main())
