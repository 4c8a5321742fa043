"""The continuous-batching server: every result matches the FP64 oracle at the
parity tolerances and is the same as the request computed alone
(single-series ls_execute), while requests of mixed sizes and precisions
arrive from several threads and share batches and streams; the device memory
the server holds (its plans' reported bytes plus its tensors) stays within its
budget."""
import threading
import time

import numpy as np
import pytest

from paper_2409_08090_gb300 import workloads as W
from tests.rerun_tolerance import assert_identical

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2409_08090_gb300 as m
    m.build.build()
    m.load_library()
    return m


def _alone(nl, s, prec, eps):
    import torch
    dev = torch.device("cuda:0")
    plan = nl.Plan(s.nd, s.nf, eps, prec)
    P = plan.execute(torch.tensor(s.t, device=dev), torch.tensor(s.y, device=dev),
                     torch.tensor(s.dy, device=dev), s.f0, s.df).cpu().numpy()
    plan.close()
    return P


def _check_oracle(oracle_mod, s, P, prec, rng, nk=384):
    # parity tolerances: FP64 at eps 1e-9 rel-l2 <= 1e-7 and max |dP| <= 1e-6;
    # FP32 at eps 1e-6 rel-l2 <= 1e-5 and max |dP| <= 1e-4 (sampled frequencies,
    # all of them for short grids)
    k = np.arange(s.nf) if s.nf <= nk else np.sort(rng.choice(s.nf, nk, replace=False))
    ref = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k)
    d = P[k] - ref
    rel = np.linalg.norm(d) / np.linalg.norm(ref)
    if prec == "fp64":
        assert np.max(np.abs(d)) <= 1e-6 and rel <= 1e-7, (s.nd, s.nf, rel)
    else:
        assert np.max(np.abs(d)) <= 1e-4 and rel <= 1e-5, (s.nd, s.nf, rel)


def test_results_in_the_mix_match_the_oracle_and_results_alone(nl, oracle_mod):
    from paper_2409_08090_gb300.serving import PeriodogramServer
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(36):
        s = W.ragged_series(1000 + i, nd_lo=50, nd_hi=4000)
        prec = "fp32" if i % 2 else "fp64"
        eps = 1e-6 if prec == "fp32" else 1e-9
        reqs.append((s, prec, eps))
    srv = PeriodogramServer(memory_budget=2 << 30, streams=2, max_batch=8)
    futs = [None] * len(reqs)

    def client(idx):
        for i in idx:
            s, prec, eps = reqs[i]
            futs[i] = srv.submit(s.t, s.y, s.dy, s.f0, s.df, s.nf, prec, eps)
            time.sleep(float(rng.exponential(0.002)))

    th = [threading.Thread(target=client, args=(list(range(k, len(reqs), 3)),)) for k in range(3)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    got = [f.result(timeout=120) for f in futs]
    stats = srv.stats()
    srv.close()
    assert stats["requests"] == len(reqs) and stats["batches"] >= 2
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    for (s, prec, eps), P in zip(reqs, got):
        assert P.shape == (s.nf,)
        _check_oracle(oracle_mod, s, P, prec, rng)
        A = _alone(nl, s, prec, eps)
        assert_identical(P, A, (s.nd, s.nf, prec))       # the same alone and in the mix


def test_device_memory_stays_within_the_budget(nl, oracle_mod):
    # Poisson-like arrivals of mixed sizes and precisions under a budget that
    # holds the four resident plans' reserved workspaces plus a few requests:
    # the high-water mark of (torch allocations + the plans' reported bytes)
    # never passes the budget, and admission still completes every request.
    import torch
    from paper_2409_08090_gb300.serving import PeriodogramServer
    rng = np.random.default_rng(9)
    budget = 1 << 30
    srv = PeriodogramServer(memory_budget=budget, streams=2, max_batch=16,
                            plan_workspace_bytes=128 << 20)
    reqs, futs = [], []
    for i in range(60):
        s = W.ragged_series(5000 + i, nd_lo=100, nd_hi=20000)
        prec = "fp32" if i % 3 else "fp64"
        reqs.append((s, prec))
        futs.append(srv.submit(s.t, s.y, s.dy, s.f0, s.df, s.nf, prec))
        time.sleep(float(rng.exponential(0.001)))
    got = [f.result(timeout=300) for f in futs]
    stats = srv.stats()
    plan_bytes = [p.device_bytes() for sl in srv.slots for p in sl.plans.values()]
    srv.close()
    assert stats["requests"] == len(reqs)
    assert plan_bytes and all(b >= 128 << 20 for b in plan_bytes)   # workspaces reserved
    assert 0 < stats["peak_device_bytes"] <= budget, stats
    torch.cuda.synchronize()
    for (s, prec), P in list(zip(reqs, got))[::6]:
        _check_oracle(oracle_mod, s, P, prec, rng, nk=128)


def test_device_results_equal_host_results(nl):
    # host results as views of the batch's pinned buffer (the default) and as
    # per-request copies (copy_limit above every batch), and device results
    import torch
    from paper_2409_08090_gb300.serving import PeriodogramServer
    reqs = [W.ragged_series(2000 + i, nd_lo=100, nd_hi=3000) for i in range(10)]
    out = {}
    for mode, limit in (("host", 0), ("host_copies", 1 << 40), ("device", 0)):
        srv = PeriodogramServer(memory_budget=2 << 30, streams=2, max_batch=4,
                                results="device" if mode == "device" else "host")
        srv.copy_limit = limit
        futs = [srv.submit(s.t, s.y, s.dy, s.f0, s.df, s.nf, "fp32", 1e-6) for s in reqs]
        out[mode] = [f.result(timeout=120) for f in futs]
        srv.close()
    for s, a, c, b in zip(reqs, out["host"], out["host_copies"], out["device"]):
        assert isinstance(b, torch.Tensor) and b.is_cuda and b.shape == (s.nf,)
        assert isinstance(a, np.ndarray) and a.shape == (s.nf,)
        assert isinstance(c, np.ndarray) and c.flags.owndata
        assert_identical(b.cpu().numpy(), a)
        assert_identical(c, a)


def test_model_variants_in_the_mix(nl):
    import torch
    from paper_2409_08090_gb300.serving import PeriodogramServer
    reqs = [W.ragged_series(3000 + i, nd_lo=100, nd_hi=2000) for i in range(6)]
    variants = [dict(normalization="psd", fit_mean=False, center_data=False),
                dict(normalization="model"), dict()]
    srv = PeriodogramServer(memory_budget=2 << 30, streams=2, max_batch=4)
    futs = [(s, v, srv.submit(s.t, s.y, s.dy, s.f0, s.df, s.nf, "fp64", 1e-9, **v))
            for s in reqs for v in variants]
    bad = srv.submit(reqs[0].t, reqs[0].y, None, 0.1, 0.1, 10, normalization="power")
    got = [(s, v, f.result(timeout=120)) for s, v, f in futs]
    srv.close()
    with pytest.raises(ValueError):
        bad.result(timeout=1)
    dev = torch.device("cuda:0")
    for s, v, P in got:
        plan = nl.Plan(s.nd, s.nf, 1e-9, "fp64")
        A = plan.execute(torch.tensor(s.t, device=dev), torch.tensor(s.y, device=dev),
                         torch.tensor(s.dy, device=dev), s.f0, s.df, **v).cpu().numpy()
        plan.close()
        assert_identical(P, A, v)


def test_invalid_and_oversized_requests_fail_their_futures_only(nl):
    from paper_2409_08090_gb300.serving import PeriodogramServer
    srv = PeriodogramServer(memory_budget=512 << 20, streams=1)
    s = W.random_case(3, 500, 2000)
    ok = srv.submit(s.t, s.y, s.dy, s.f0, s.df, s.nf, "fp64", 1e-9)
    bad = srv.submit(s.t, s.y * np.nan, s.dy, s.f0, s.df, s.nf)
    big = srv.submit(s.t, s.y, s.dy, s.f0, s.df, 50_000_000)     # grids beyond a plan lane
    with pytest.raises(ValueError):
        bad.result(timeout=60)
    with pytest.raises(MemoryError):
        big.result(timeout=60)
    P = ok.result(timeout=60)
    srv.close()
    assert_identical(P, _alone(nl, s, "fp64", 1e-9))
