"""Serving form on the GPU: a small complex k-point/SCF stream through the continuous-batching
server.  Each result computed in the mix must be the one computed alone (bit for bit: the
kernels are deterministic and every request runs on its own handle), factor reuse must match a
fresh factorisation, and every eigenvalue must match the oracle to 1e-11 ||H||_1."""
import numpy as np
import pytest

import oracle
from paper_2502_02460_gb300 import inputs
from tests.pins import norm1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch

    from paper_2502_02460_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def scf_inputs(n, sid, iters, cx=True):
    p = inputs.make_problem(n, max(1, n // 4), seed=4000 + sid, complex_=cx)
    out = []
    for t in range(iters):
        rng = np.random.default_rng(5000 + 1000 * sid + t)
        G = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cx else 0)
        dH = 0.5 * (G + G.conj().T)
        H = p.H + (1e-3 * np.linalg.norm(p.H) / np.linalg.norm(dH) * dH if t > 0 else 0)
        out.append(H)
    return p.S, out


def test_stream_results_in_the_mix_equal_results_alone(dev):
    import torch

    from paper_2502_02460_gb300 import gev, serve

    sizes = {0: 96, 1: 150, 2: 64, 3: 200}
    iters = 3
    data = {sid: scf_inputs(n, sid, iters) for sid, n in sizes.items()}
    srv = serve.Server(budget_bytes=40e9, workers=4, device=dev)
    futs = {}
    for t in range(iters):  # interleaved arrivals of the systems' SCF iterations
        for sid, n in sizes.items():
            S, Hs = data[sid]
            k = max(1, n // 4)
            Sb = gev.cm_from_numpy(S, dev) if t == 0 else None
            futs[(sid, t)] = srv.submit(sid, gev.cm_from_numpy(Hs[t], dev), Sb, k, n=n, complex_=True,
                                        last=(t == iters - 1))
    res = {key: f.result(timeout=300) for key, f in futs.items()}
    srv.close()
    st = srv.stats()
    assert st["requests"] == len(futs) and st["factor_reuses"] == len(sizes) * (iters - 1)
    for (sid, t), (w, Cb, rep) in res.items():
        n = sizes[sid]
        k = max(1, n // 4)
        S, Hs = data[sid]
        with gev.Solver(n, complex_=True, device=dev) as s:  # alone, fresh factor
            wa, Ca = s.solve_cm(gev.cm_from_numpy(Hs[t], dev), gev.cm_from_numpy(S, dev), k)
        assert torch.equal(w, wa) and torch.equal(Cb, Ca), (sid, t)
        wo, _, info, _ = oracle.gev(Hs[t], S, k)
        assert np.max(np.abs(w.cpu().numpy() - wo)) <= 1e-11 * norm1(Hs[t])


def test_mixed_stream_results_in_the_mix_equal_results_alone(dev):
    """The serving form in mixed precision (complex pencils through the mixed form): each result in
    the mix equals the result computed alone, bit for bit, and meets the oracle's eigenvalue bound."""
    import torch

    from paper_2502_02460_gb300 import gev, serve

    sizes = {0: 120, 1: 64, 2: 180}
    iters = 2
    data = {sid: scf_inputs(n, sid, iters) for sid, n in sizes.items()}
    srv = serve.Server(budget_bytes=40e9, workers=3, device=dev, mixed=True)
    futs = {}
    for t in range(iters):
        for sid, n in sizes.items():
            S, Hs = data[sid]
            k = max(1, n // 4)
            Sb = gev.cm_from_numpy(S, dev) if t == 0 else None
            futs[(sid, t)] = srv.submit(sid, gev.cm_from_numpy(Hs[t], dev), Sb, k, n=n, complex_=True,
                                        last=(t == iters - 1))
    res = {key: f.result(timeout=300) for key, f in futs.items()}
    srv.close()
    for (sid, t), (w, Cb, rep) in res.items():
        n = sizes[sid]
        k = max(1, n // 4)
        S, Hs = data[sid]
        with gev.Solver(n, complex_=True, device=dev, mixed=True) as s:
            wa, Ca = s.solve_cm(gev.cm_from_numpy(Hs[t], dev), gev.cm_from_numpy(S, dev), k)
        assert torch.equal(w, wa) and torch.equal(Cb, Ca), (sid, t)
        wo, _, info, _ = oracle.gev(Hs[t], S, k)
        assert np.max(np.abs(w.cpu().numpy() - wo)) <= 1e-11 * norm1(Hs[t])
