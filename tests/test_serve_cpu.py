"""Host-side logic of the serving form (no GPU): admission under the memory budget, SCF ordering
per system, overlap of different systems, failure isolation, the stream plan, and the split of the
stream over replicas (world_size 2, gloo) with no collective on the data path."""
import threading
import time

import pytest

from paper_2502_02460_gb300 import serve


class FakeGPU:
    """Stands in for the handles: records concurrency and call order."""

    def __init__(self, delay=0.01, fail_on=None):
        self.delay = delay
        self.fail_on = fail_on or set()
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.calls = []
        self.live_handles = 0

    def make(self, n, cx):
        with self.lock:
            self.live_handles += 1
        return {"n": n}

    def free(self, h):
        with self.lock:
            self.live_handles -= 1

    def solve(self, h, req):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.calls.append((req.system_id, req.H))
        time.sleep(self.delay)
        with self.lock:
            self.active -= 1
        if (req.system_id, req.H) in self.fail_on:
            raise RuntimeError("GEV_ERR_NOT_SPD")
        return ("result", req.system_id, req.H)


def make_server(fake, budget, workers=4, per_system=10):
    return serve.Server(budget_bytes=budget, workers=workers, solve_fn=fake.solve,
                        bytes_fn=lambda n, cx: per_system, make_handle=fake.make, free_handle=fake.free)


def test_scf_iterations_of_a_system_run_in_order_and_systems_overlap():
    fake = FakeGPU(delay=0.02)
    srv = make_server(fake, budget=1000)
    futs = []
    for it in range(4):
        for sid in range(3):
            futs.append((sid, it, srv.submit(sid, it, None, 1, n=8, complex_=True, last=(it == 3))))
    for sid, it, f in futs:
        assert f.result(timeout=10) == ("result", sid, it)
    srv.close()
    for sid in range(3):
        its = [h for (s, h) in fake.calls if s == sid]
        assert its == sorted(its)
    assert fake.max_active >= 2  # different systems ran concurrently
    assert fake.live_handles == 0
    st = srv.stats()
    assert st["requests"] == 12 and st["p99_ms"] >= st["p50_ms"] > 0


def test_admission_respects_the_budget():
    fake = FakeGPU(delay=0.01)
    srv = make_server(fake, budget=25, per_system=10)  # at most two live systems
    futs = [srv.submit(sid, 0, None, 1, n=8, complex_=True, last=True) for sid in range(6)]
    for f in futs:
        f.result(timeout=10)
    srv.close()
    assert srv.peak_bytes <= 25
    assert fake.max_active <= 2


def test_request_larger_than_budget_is_rejected_others_served():
    fake = FakeGPU()
    srv = serve.Server(budget_bytes=100, workers=2, solve_fn=fake.solve,
                       bytes_fn=lambda n, cx: 1000 if n > 100 else 10, make_handle=fake.make,
                       free_handle=fake.free)
    big = srv.submit("big", 0, None, 1, n=500, complex_=False, last=True)
    small = srv.submit("small", 0, None, 1, n=50, complex_=False, last=True)
    assert small.result(timeout=10)[0] == "result"
    with pytest.raises(MemoryError):
        big.result(timeout=10)
    srv.close()
    assert srv.rejected == 1


def test_a_failing_request_does_not_affect_the_others():
    fake = FakeGPU(fail_on={(1, 0)})
    srv = make_server(fake, budget=1000)
    f_bad = srv.submit(1, 0, None, 1, n=8, complex_=True)
    f_good = [srv.submit(s, 0, None, 1, n=8, complex_=True, last=True) for s in (2, 3)]
    with pytest.raises(RuntimeError):
        f_bad.result(timeout=10)
    for f in f_good:
        assert f.result(timeout=10)[0] == "result"
    srv.close()


def test_stream_plan_matches_the_recipe():
    spec = serve.StreamSpec()
    plan = serve.stream_plan(spec)
    assert len(plan) == 512
    times = [p[0] for p in plan]
    assert all(b > a for a, b in zip(times, times[1:]))
    assert 1.5 < times[-1] < 4.0  # mean inter-arrival 5 ms
    sizes = {p[1]: p[3] for p in plan}
    assert len(sizes) == 52 and min(sizes.values()) >= 256 and max(sizes.values()) <= 8192
    assert all(p[4] == -(-p[3] // 4) for p in plan)  # k = ceil(0.25 N)
    last_sys = [p for p in plan if p[1] == 51]
    assert len(last_sys) == 2 and last_sys[-1][5]


def _replica(rank, world, out):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:29517", rank=rank, world_size=world)
    plan = serve.stream_plan(serve.StreamSpec(requests=40, scf_iters=10))
    mine = [p for p in plan if p[1] % world == rank]  # systems pinned to replicas by id
    fake = FakeGPU(delay=0.001)
    srv = make_server(fake, budget=1000)
    futs = [srv.submit(p[1], p[2], None, p[4], n=p[3], complex_=True, last=p[5]) for p in mine]
    for f in futs:
        f.result(timeout=30)
    srv.close()
    import torch

    t = torch.tensor([len(mine)])
    dist.all_reduce(t)  # bookkeeping only (count of served requests), not on the data path
    out[rank] = int(t.item())
    dist.destroy_process_group()


def test_stream_splits_over_two_replicas():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_replica, args=(r, 2, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert out[0] == out[1] == 40
