"""Ragged batches through ls_execute_batch: every series must match the oracle
at the single-series tolerances and the single-series path (ls_execute) at
rounding level, however the batch is grouped into launches."""
import numpy as np
import pytest

from paper_2409_08090_gb300 import workloads as W
from tests.rerun_tolerance import assert_identical, assert_rerun_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2409_08090_gb300 as m
    m.build.build()
    m.load_library()
    return m


def _series(seed, n=14):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nd = int(rng.choice([40, 300, 1000, 2500, 5000]))
        nf = int(rng.choice([1, 7, 500, 3000, 9001, 20000]))
        s = W.random_case(seed * 100 + i, nd, nf, sort=bool(i % 2), unit_dy=(i % 3 == 0),
                          df_t=float(rng.choice([0.2, 0.9, 1.7])),
                          baseline=float(rng.uniform(10, 500)))
        out.append(s)
    return out


def _pack(series):
    import torch
    dev = torch.device("cuda:0")
    offsets = np.zeros(len(series) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([s.nd for s in series])
    t = torch.tensor(np.concatenate([s.t for s in series]), device=dev)
    y = torch.tensor(np.concatenate([s.y for s in series]), device=dev)
    dyv = [np.ones(s.nd) if s.dy is None else s.dy for s in series]
    dy = torch.tensor(np.concatenate(dyv), device=dev)
    return offsets, t, y, dy


def _run_batch(nl, series, eps, prec, budget=0):
    offsets, t, y, dy = _pack(series)
    plan = nl.Plan(2, 1, eps, prec, batch_workspace_bytes=budget)
    P, off = plan.execute_batch(t, y, dy, offsets, [s.f0 for s in series],
                                [s.df for s in series], [s.nf for s in series])
    P = P.cpu().numpy()
    plan.close()
    return [P[o:o + s.nf] for o, s in zip(off, series)]


def _run_single(nl, s, eps, prec):
    import torch
    dev = torch.device("cuda:0")
    plan = nl.Plan(s.nd, s.nf, eps, prec)
    dy = torch.tensor(np.ones(s.nd) if s.dy is None else s.dy, device=dev)
    P = plan.execute(torch.tensor(s.t, device=dev), torch.tensor(s.y, device=dev), dy,
                     s.f0, s.df).cpu().numpy()
    plan.close()
    return P


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_ragged_batch_matches_oracle_and_single(nl, oracle_mod, prec, eps):
    series = _series(3)
    got = _run_batch(nl, series, eps, prec)
    for s, P in zip(series, got):
        P_o = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, np.arange(s.nf))
        assert np.all(np.isfinite(P))
        if prec == "fp64":
            assert np.max(np.abs(P - P_o)) <= 1e-9
        else:
            assert np.max(np.abs(P - P_o)) <= 1e-4
            # relative l2 is the FP32 bar for a periodogram; over one or a few
            # small values it is their relative error, which FP32 sums
            # (rounding ~1e-7 of sum |h|) cannot bound at P ~ 1e-4
            if s.nd >= 500 and s.nf >= 100:
                assert np.linalg.norm(P - P_o) / np.linalg.norm(P_o) <= 1e-5
        P_1 = _run_single(nl, s, eps, prec)
        assert_identical(P, P_1, (s.nd, s.nf))


def test_small_budget_splits_launches_without_changing_results(nl):
    series = _series(5, n=10)
    full = _run_batch(nl, series, 1e-9, "fp64")
    split = _run_batch(nl, series, 1e-9, "fp64", budget=2_000_000)
    for a, b in zip(full, split):
        assert np.max(np.abs(a - b)) <= 1e-12


def test_shared_times_uniform_batch(nl, oracle_mod):
    # the uniform-batch shape: many series on one time array (replicated here)
    t, Y, dy, f0, df, nf = W.uniform_batch(nseries=48, nd=2000, nf=24_000)
    series = [W.Series(t, Y[i], dy, f0, df, nf) for i in range(Y.shape[0])]
    got = _run_batch(nl, series, 1e-6, "fp32")
    for i in (0, 17, 47):
        s = series[i]
        P_o = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, np.arange(nf))
        assert np.linalg.norm(got[i] - P_o) / np.linalg.norm(P_o) <= 1e-5


def test_bad_series_is_reported_at_sync(nl):
    import torch
    series = _series(7, n=4)
    series[2].y = series[2].y.copy()
    series[2].y[1] = np.nan
    offsets, t, y, dy = _pack(series)
    plan = nl.Plan(2, 1, 1e-9, "fp64")
    with pytest.raises(nl.LSError) as ei:
        plan.execute_batch(t, y, dy, offsets, [s.f0 for s in series], [s.df for s in series],
                           [s.nf for s in series])
    assert ei.value.status == nl.LS_ERR_ARG
    # invalid metadata is rejected before any launch
    with pytest.raises(nl.LSError):
        plan.execute_batch(t, y, dy, offsets, [s.f0 for s in series], [-1.0] * 4,
                           [s.nf for s in series])
    plan.close()


def test_two_point_series_in_a_batch(nl, oracle_mod):
    # Two points fit a sinusoid plus offset exactly: P = 1 wherever the normal
    # matrix is well conditioned (its non-zero eigenvalue clearly above the sums'
    # accuracy); elsewhere the value is not determined to the tolerance and only
    # has to be a valid power.
    series = [W.random_case(900 + i, 2, 4000, baseline=50.0) for i in range(6)]
    for prec, eps in (("fp64", 1e-12), ("fp32", 1e-6)):
        got = _run_batch(nl, series, eps, prec)
        for s, P in zip(series, got):
            _, S = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, np.arange(s.nf),
                                          return_sums=True)
            C, Sn, C2 = S[:, 2], S[:, 3], S[:, 4]
            trace = (0.5 * (1 + C2) - C * C) + (0.5 * (1 - C2) - Sn * Sn)   # = the eigenvalue
            ok = trace > 1e4 * max(eps, 1e-7)
            assert ok.mean() > 0.5
            assert np.max(np.abs(P[ok] - 1.0)) <= (1e-8 if prec == "fp64" else 1e-3)
            # near-singular frequencies: error ~ (sums' accuracy) / eigenvalue
            assert np.all(np.isfinite(P)) and P.min() >= -1e-6 and P.max() <= 1.1


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-6), ("fp64", 1e-12)])
def test_shared_times_batch_matches_replicated_batch(nl, oracle_mod, prec, eps):
    import torch
    t, Y, dy, f0, df, nf = W.uniform_batch(seed=11, nseries=40, nd=1500, nf=9000)
    dev = torch.device("cuda:0")
    plan = nl.Plan(2, 1, eps, prec, batch_workspace_bytes=3_000_000)   # several launches
    Pshared = plan.execute_shared(torch.tensor(t, device=dev), torch.tensor(Y, device=dev),
                                  torch.tensor(dy, device=dev), f0, df, nf).cpu().numpy()
    plan.close()
    series = [W.Series(t, Y[i], dy, f0, df, nf) for i in range(Y.shape[0])]
    Prep = _run_batch(nl, series, eps, prec)
    for i in range(Y.shape[0]):
        assert_rerun_close(Pshared[i], Prep[i], prec)
    for i in (0, 39):
        P_o = oracle_mod.periodogram(t, Y[i], dy, f0, df, np.arange(nf))
        if prec == "fp64":
            assert np.max(np.abs(Pshared[i] - P_o)) <= 1e-9
        else:
            assert np.linalg.norm(Pshared[i] - P_o) / np.linalg.norm(P_o) <= 1e-5


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-6), ("fp64", 1e-9)])
def test_series_same_bits_alone_and_in_a_wide_batch(nl, prec, eps):
    # 300 series share one launch, so each gets few reduction blocks, against
    # many alone: the FP64 sums go per fixed chunk of points, so the launch
    # shape cannot change a series' bits
    rng = np.random.default_rng(17)
    series = []
    for i in range(300):
        nd = int(rng.integers(1500, 6000))
        t = np.sort(rng.uniform(0.0, 500.0, nd))
        y = np.sin(2 * np.pi * t / rng.uniform(0.5, 50.0)) + rng.normal(0.0, 1.0, nd)
        dy = rng.uniform(0.5, 2.0, nd)
        series.append(W.Series(t, y, dy, 1e-3, 1e-3, 3000 + 7 * i))
    got = _run_batch(nl, series, eps, prec)
    for i in (0, 149, 299):
        assert_identical(got[i], _run_single(nl, series[i], eps, prec), i)


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-6), ("fp64", 1e-9)])
def test_shared_times_series_same_bits_alone_and_in_the_batch(nl, prec, eps):
    # a series of a shared-times batch gives the same bits in a shared-times
    # batch of its own and when the batch is cut into several launches: the
    # common transforms are recomputed identically and each series keeps its
    # own fixed-point grids whatever the grouping
    import torch
    t, Y, dy, f0, df, nf = W.uniform_batch(seed=12, nseries=24, nd=1200, nf=7000)
    dev = torch.device("cuda:0")
    tt, yy, dd = (torch.tensor(a, device=dev) for a in (t, Y, dy))
    plan = nl.Plan(2, 1, eps, prec)
    P = plan.execute_shared(tt, yy, dd, f0, df, nf).cpu().numpy()
    small = nl.Plan(2, 1, eps, prec, batch_workspace_bytes=3_000_000)
    Psplit = small.execute_shared(tt, yy, dd, f0, df, nf).cpu().numpy()
    for i in (0, 11, 23):
        Pi = plan.execute_shared(tt, yy[i:i + 1].contiguous(), dd, f0, df, nf).cpu().numpy()[0]
        assert_identical(P[i], Pi, i)
    plan.close()
    small.close()
    assert_identical(P, Psplit)
