"""Autotuner of the band width b of the two-stage tridiagonalisation (which is also the panel width of
the one-stage route; each timed solve takes the route ``gev_opts.one_stage = 0`` picks automatically).

The full -> band step gains from a wide band (its products have inner dimension b), the bulge chasing
and back-transform 2 lose from it (a band -> tridiagonal task costs ~6 b^2 flops on a 3n-task
critical path), and the balance moves with the dtype, the order n and the precision form.  The
tuner times complete solves (``gev_solve``, CUDA events on the solve stream, inputs resident) of the
seeded synthetic pencils for every candidate b and keeps the fastest per (dtype, order bucket,
precision); ``Solver(band_b=0)`` then takes the table's entry for its bucket (the nearest tuned order
at or below n, else the smallest).  b = 128 is not a candidate: the bulge-chasing kernel stages three
b x b blocks of the band in shared memory (3 x 128 x 129 x 8 B = 396 KB > the 227 KB of a CTA).

    python -m paper_2502_02460_gb300.tune [--orders 1024 2048 4096 8192] [--reps 2] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuned_band.json")
CANDIDATES = (16, 32, 64)

_table = None


def key(complex_: bool, mixed: bool) -> str:
    return ("c128" if complex_ else "f64") + ("/mixed" if mixed else "/plain")


def load(path: str = TABLE) -> dict:
    global _table
    if _table is None:
        try:
            with open(path) as f:
                _table = json.load(f)
        except (OSError, ValueError):
            _table = {}
    return _table


def pick_band(n: int, complex_: bool, mixed: bool, table: dict | None = None) -> int:
    """The tuned band width for a problem of order n (0 when the table has no entry: the library's
    default)."""
    t = (table if table is not None else load()).get("entries", {}).get(key(complex_, mixed), {})
    if not t:
        return 0
    orders = sorted(int(o) for o in t)
    below = [o for o in orders if o <= n]
    o = below[-1] if below else orders[0]
    return int(t[str(o)]["b"])


def time_solve(n: int, complex_: bool, mixed: bool, b: int, reps: int, dev) -> dict:
    import torch

    from . import gev, inputs

    k = max(1, n // 4)
    on_gpu = n > 4096
    p = inputs.make_problem(n, k, seed=11, complex_=complex_, device=dev if on_gpu else None, gap_check=False)
    Hb, Sb = (p.H, p.S) if on_gpu else (gev.cm_from_numpy(p.H, dev), gev.cm_from_numpy(p.S, dev))
    stream = torch.cuda.current_stream(dev)
    with gev.Solver(n, complex_=complex_, device=dev, mixed=mixed, band_b=b, timing=1, stream=stream) as s:
        w = torch.empty(k, dtype=torch.float64, device=dev)
        Cb = torch.empty((k, n), dtype=s.dtype, device=dev)
        s.solve_cm(Hb, Sb, k, w, Cb)  # warm-up
        times = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.solve_cm(Hb, Sb, k, w, Cb)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        steps = s.last_report["ms"]
    return {"ms": statistics.median(times), "steps_ms": steps}


def tune(orders, reps: int, dev, forms=((False, False), (False, True), (True, False), (True, True))) -> dict:
    entries = {}
    for complex_, mixed in forms:
        kk = key(complex_, mixed)
        for n in orders:
            res = {b: time_solve(n, complex_, mixed, b, reps, dev) for b in CANDIDATES}
            best = min(res, key=lambda b: res[b]["ms"])
            entries.setdefault(kk, {})[str(n)] = {"b": best, "ms": {str(b): round(r["ms"], 2) for b, r in res.items()}}
            print(kk, n, {b: round(r["ms"], 1) for b, r in res.items()}, "->", best, flush=True)
    return entries


def main():
    import torch

    from . import build

    ap = argparse.ArgumentParser()
    ap.add_argument("--orders", type=int, nargs="+", default=[1024, 2048, 4096, 8192])
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--out", default=TABLE)
    args = ap.parse_args()
    build.build()
    dev = torch.device("cuda", 0)
    t0 = time.time()
    entries = tune(args.orders, args.reps, dev)
    table = {"what": "band width b of the two-stage tridiagonalisation (panel width of the one-stage route), "
                     "fastest complete solve (k = n/4, automatic route) of the seeded synthetic pencil, per "
                     "dtype/precision and order",
             "candidates": list(CANDIDATES), "reps": args.reps, "gpu": torch.cuda.get_device_name(dev),
             "tuning_s": round(time.time() - t0, 1), "entries": entries}
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
