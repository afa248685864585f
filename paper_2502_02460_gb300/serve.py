"""Serving form: continuous batching of independent generalized eigenproblems.

ELSI's trivially parallel handling of k-points and spin channels (section "ELSI", Figure 1 caption)
and FHI-aims' SCF cycle turn one material into a stream of independent solves: every system
(k-point / spin channel) recurs once per SCF iteration with a new H and the same S.  The server

* keeps one solver handle per live system, with its own CUDA stream and the system's inverted
  Cholesky factor resident across SCF iterations (the first request of a system passes S, later
  ones may pass S=None and skip Cholesky and inversion);
* admits requests as they arrive and as slots and device memory free up (a system's handle is
  created only when its workspace fits the budget next to the live ones) - continuous batching:
  requests never wait for a batch to fill or drain, and different systems' solves run
  concurrently on their own streams (worker threads call the C ABI with the GIL released);
* serves a system's SCF iterations in order (iteration t after t-1: t reuses t-1's factor);
* records the latency of every request from its arrival to its result (p50/p99) and solves/s.

Each result depends only on its own inputs (the kernels are deterministic and a request runs on its
own handle), so a result computed inside the mix is bit-for-bit the one computed alone.

The scheduling logic is independent of the GPU: ``solve_fn`` and ``bytes_fn`` can be replaced (the
CPU tests use fakes); by default they are the library's handles.
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import threading
import time
from typing import Callable, Optional


@dataclasses.dataclass
class Request:
    system_id: object
    H: object
    S: object
    k: int
    n: int
    complex_: bool
    arrival: float
    last: bool
    future: concurrent.futures.Future
    seq: int = 0
    start: float = 0.0
    end: float = 0.0


class _System:
    def __init__(self, sid, n, complex_):
        self.sid = sid
        self.n = n
        self.complex_ = complex_
        self.queue = collections.deque()
        self.busy = False
        self.handle = None
        self.bytes = 0
        self.done = 0
        self.finished = False


def default_bytes_fn(n: int, complex_: bool, mixed: bool) -> int:
    import ctypes

    from . import gev

    o = gev.Opts()
    gev.lib().gev_default_opts(ctypes.byref(o))
    o.prec = gev.GEV_MIXED if mixed else gev.GEV_PLAIN
    return int(gev.lib().gev_workspace_bytes(n, gev.GEV_C128 if complex_ else gev.GEV_F64, ctypes.byref(o)))


class Server:
    """Continuous-batching server over the C ABI (see the module docstring).

    submit(system_id, H, S, k, last=False) -> Future resolving to (eigenvalues, C) as torch tensors
    (column-major buffers, see gev.py).  H, S are column-major device buffers (S=None to reuse the
    system's resident factor).  ``last=True`` on a system's final request frees its handle after
    the solve.
    """

    def __init__(self, budget_bytes: float = 120e9, mixed: bool = False, workers: int = 4, device=None,
                 solve_fn: Optional[Callable] = None, bytes_fn: Optional[Callable] = None,
                 make_handle: Optional[Callable] = None, free_handle: Optional[Callable] = None):
        self.budget = float(budget_bytes)
        self.mixed = mixed
        self.device = device
        self._solve_fn = solve_fn or self._gpu_solve
        self._bytes_fn = bytes_fn or (lambda n, cx: default_bytes_fn(n, cx, mixed))
        self._make_handle = make_handle or self._gpu_handle
        self._free_handle = free_handle or (lambda h: h.close())
        self._cv = threading.Condition()
        self._systems: dict = {}
        self._order = collections.deque()  # arrival order of pending requests' systems
        self._inflight_bytes = 0
        self._closed = False
        self._seq = 0
        self.completed: list = []
        self.rejected = 0
        self.peak_bytes = 0
        self.factor_reuses = 0
        self._t0 = None
        self._threads = [threading.Thread(target=self._worker, daemon=True) for _ in range(workers)]
        for t in self._threads:
            t.start()

    # ------------------------------------------------------------------------------- public --
    def submit(self, system_id, H, S, k: int, n: int = None, complex_: bool = None, last: bool = False,
               arrival: float = None) -> concurrent.futures.Future:
        fut = concurrent.futures.Future()
        n = n if n is not None else H.shape[0]
        if complex_ is None:
            complex_ = bool(getattr(H, "is_complex", lambda: False)())
        now = time.perf_counter()
        req = Request(system_id, H, S, k, n, complex_, arrival if arrival is not None else now, last, fut)
        with self._cv:
            if self._closed:
                raise RuntimeError("server closed")
            if self._t0 is None:
                self._t0 = req.arrival
            req.seq = self._seq
            self._seq += 1
            sysm = self._systems.get(system_id)
            if sysm is None:
                sysm = _System(system_id, n, complex_)
                self._systems[system_id] = sysm
            sysm.queue.append(req)
            self._order.append(system_id)
            self._cv.notify_all()
        return fut

    def close(self, wait: bool = True):
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        if wait:
            for t in self._threads:
                t.join()
        for sysm in list(self._systems.values()):
            if sysm.handle is not None:
                self._free_handle(sysm.handle)
                sysm.handle = None

    def drain(self):
        """Block until every submitted request has completed."""
        with self._cv:
            while any(s.queue or s.busy for s in self._systems.values()):
                self._cv.wait(0.05)

    def stats(self) -> dict:
        lat = sorted((r.end - r.arrival) * 1e3 for r in self.completed)
        if not lat:
            return {"requests": 0}
        pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
        span = max(r.end for r in self.completed) - min(r.arrival for r in self.completed)
        return {"requests": len(lat), "p50_ms": pct(0.50), "p99_ms": pct(0.99), "max_ms": lat[-1],
                "solves_per_s": len(lat) / span if span > 0 else None,
                "peak_admitted_bytes": self.peak_bytes, "factor_reuses": self.factor_reuses,
                "rejected": self.rejected}

    # ----------------------------------------------------------------------------- internals --
    def _gpu_handle(self, n, complex_):
        from . import gev

        import torch

        stream = torch.cuda.Stream(device=self.device)
        h = gev.Solver(n, complex_=complex_, device=self.device, mixed=self.mixed, stream=stream)
        h.reuse_factor(True)
        return h

    @staticmethod
    def _gpu_solve(handle, req):
        import torch

        with torch.cuda.stream(handle.stream):
            w, Cb = handle.solve_cm(req.H, req.S, req.k)
        handle.stream.synchronize()
        return w, Cb, handle.last_report

    def _pick(self):
        """Earliest-arrived request whose system is idle and whose handle exists or fits."""
        for sid in list(self._order):
            sysm = self._systems[sid]
            if sysm.busy or not sysm.queue:
                continue
            if sysm.handle is None:
                need = self._bytes_fn(sysm.n, sysm.complex_)
                if need > self.budget:
                    return sysm, "reject"
                if self._inflight_bytes + need > self.budget:
                    continue  # wait for memory; later arrivals of live systems may still run
                sysm.bytes = need
                self._inflight_bytes += need
                self.peak_bytes = max(self.peak_bytes, self._inflight_bytes)
                sysm.handle = "pending"
            return sysm, "run"
        return None, None

    def _worker(self):
        while True:
            with self._cv:
                while True:
                    if self._closed and not any(s.queue for s in self._systems.values()):
                        return
                    sysm, what = self._pick()
                    if sysm is not None:
                        break
                    self._cv.wait(0.05)
                req = sysm.queue.popleft()
                self._order.remove(sysm.sid)
                if what == "reject":
                    self.rejected += 1
                    req.future.set_exception(MemoryError(f"system {sysm.sid}: workspace exceeds the budget"))
                    continue
                sysm.busy = True
                need_handle = sysm.handle == "pending"
            try:
                if need_handle:
                    sysm.handle = self._make_handle(sysm.n, sysm.complex_)
                req.start = time.perf_counter()
                if req.S is None:
                    self.factor_reuses += 1
                out = self._solve_fn(sysm.handle, req)
                req.end = time.perf_counter()
                req.future.set_result(out)
                ok = True
            except BaseException as exc:  # the request fails, the others go on
                req.end = time.perf_counter()
                req.future.set_exception(exc)
                ok = False
            with self._cv:
                sysm.busy = False
                sysm.done += 1
                if ok:
                    self.completed.append(req)
                if req.last or (not ok and sysm.handle not in (None, "pending") and not sysm.queue):
                    if sysm.handle not in (None, "pending"):
                        self._free_handle(sysm.handle)
                    sysm.handle = None
                    self._inflight_bytes -= sysm.bytes
                    sysm.bytes = 0
                    sysm.finished = req.last
                self._cv.notify_all()


# ------------------------------------------------------------------------------ the workload --
@dataclasses.dataclass
class StreamSpec:
    requests: int = 512
    rate_hz: float = 200.0
    n_min: int = 256
    n_max: int = 8192
    scf_iters: int = 10
    k_frac: float = 0.25
    dh_rel: float = 1e-3
    complex_: bool = True


def stream_plan(spec: StreamSpec, seed_arrivals: int = 40, seed_sizes: int = 41):
    """(arrival time, system id, SCF iteration, n, k) for every request of the k-point stream:
    Poisson arrivals, systems of log-uniform size recurring for scf_iters iterations (the last
    system truncated), iteration t of a system after t-1."""
    import math

    import numpy as np

    ra = np.random.default_rng(seed_arrivals)
    rs = np.random.default_rng(seed_sizes)
    nsys = (spec.requests + spec.scf_iters - 1) // spec.scf_iters
    sizes = [int(round(math.exp(rs.uniform(math.log(spec.n_min), math.log(spec.n_max))))) for _ in range(nsys)]
    t = 0.0
    plan = []
    for r in range(spec.requests):
        t += ra.exponential(1.0 / spec.rate_hz)
        sid, it = r // spec.scf_iters, r % spec.scf_iters
        n = sizes[sid]
        k = max(1, int(math.ceil(spec.k_frac * n)))
        last = (it == spec.scf_iters - 1) or (r == spec.requests - 1)
        plan.append((t, sid, it, n, k, last))
    return plan
