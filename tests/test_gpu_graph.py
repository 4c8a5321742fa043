"""CUDA-graph replay of ls_execute: a recorded pipeline re-run on new contents
of the same device buffers gives the same result as a direct call."""
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


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_graph_replay_matches_direct_calls(nl, oracle_mod, prec, eps):
    import torch
    dev = torch.device("cuda:0")
    cases = [W.random_case(300 + i, 1500, 6000, baseline=150.0) for i in range(3)]
    t = torch.tensor(cases[0].t, device=dev)
    y = torch.tensor(cases[0].y, device=dev)
    dy = torch.tensor(cases[0].dy, device=dev)
    s0 = cases[0]
    plan = nl.Plan(s0.nd, s0.nf, eps, prec)
    g = plan.graph(t, y, dy, s0.f0, s0.df)
    for s in cases:
        t.copy_(torch.tensor(s.t))
        y.copy_(torch.tensor(s.y))
        dy.copy_(torch.tensor(s.dy))
        P = g.replay().clone()
        g.sync()
        ref_plan = nl.Plan(s.nd, s.nf, eps, prec)
        direct = ref_plan.execute(torch.tensor(s.t, device=dev), torch.tensor(s.y, device=dev),
                                  torch.tensor(s.dy, device=dev), s0.f0, s0.df).cpu().numpy()
        ref_plan.close()
        assert_identical(P.cpu().numpy(), direct)
        # the graph keeps the recorded grid (f0, df of the first case)
        k = np.arange(0, s.nf, 97)
        P_o = oracle_mod.periodogram(s.t, s.y, s.dy, s0.f0, s0.df, k)
        tol = 1e-9 if prec == "fp64" else 1e-4
        assert np.max(np.abs(P.cpu().numpy()[k] - P_o)) <= tol
    plan.close()


def test_graph_reports_device_errors_at_sync(nl):
    import torch
    dev = torch.device("cuda:0")
    s = W.random_case(310, 500, 2000)
    t, y, dy = (torch.tensor(a, device=dev) for a in (s.t, s.y, s.dy))
    plan = nl.Plan(s.nd, s.nf, 1e-9, "fp64")
    g = plan.graph(t, y, dy, s.f0, s.df)
    y[3] = float("nan")
    g.replay()
    with pytest.raises(nl.LSError):
        g.sync()
    y[3] = 0.5
    g.replay()
    g.sync()
    plan.close()


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-6), ("fp64", 1e-9)])
def test_tuned_plan_matches_the_oracle(nl, oracle_mod, tmp_path, monkeypatch, prec, eps):
    # the autotuner measures its 8 configurations on the device; the plan built
    # from the cached entry takes them and still meets the tolerance
    import torch
    from paper_2409_08090_gb300 import autotune
    monkeypatch.setenv("LS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    s = W.random_case(320, 3000, 30_000, baseline=300.0)
    e = autotune.tune(s.nf, eps, prec, nd=s.nd, reps=3)
    assert e["upsampling"] in autotune.CANDIDATES and len(e["ms"]) >= 4
    plan = nl.Plan(s.nd, s.nf, eps, prec, upsampling="tuned")
    assert abs(plan.info.sigma - e["upsampling"]) < 1e-12
    if e["cols_per_block"]:
        assert plan.info.cols_per_block in (e["cols_per_block"], 1, 2, 4, 8)
    dev = torch.device("cuda:0")
    P = plan.execute(torch.tensor(s.t, device=dev), torch.tensor(s.y, device=dev),
                     torch.tensor(s.dy, device=dev), s.f0, s.df).cpu().numpy()
    plan.close()
    P_o = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, np.arange(s.nf))
    if prec == "fp64":
        assert np.max(np.abs(P - P_o)) <= 1e-6
    else:
        assert np.linalg.norm(P - P_o) / np.linalg.norm(P_o) <= 1e-5
