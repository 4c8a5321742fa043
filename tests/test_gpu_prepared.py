"""Prepared batches (ls_batch_prepare / ls_batch_run) and their CUDA-graph
replay: a prepared run gives the periodograms of ls_execute_batch (to the
rounding of the spread's atomic additions) for every new set of values in the
layout, also when the budget cuts the batch into several launches, and a
recorded graph replays the whole batch on the current contents of its
inputs."""
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


def _dev(a):
    import torch
    return torch.tensor(a, device="cuda:0")


def _ragged(seed, n=12):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nd = int(rng.choice([60, 400, 1500, 4000]))
        nf = int(rng.choice([5, 300, 2500, 9001]))
        out.append(W.random_case(seed * 100 + i, nd, nf, unit_dy=(i % 4 == 0),
                                 df_t=float(rng.choice([0.2, 0.8])),
                                 baseline=float(rng.uniform(20, 400))))
    return out


def _layout(series):
    offsets = np.zeros(len(series) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([s.nd for s in series])
    t = _dev(np.concatenate([s.t for s in series]))
    dy = _dev(np.concatenate([np.ones(s.nd) if s.dy is None else s.dy for s in series]))
    return offsets, t, dy


def _grids(series):
    return [s.f0 for s in series], [s.df for s in series], [s.nf for s in series]


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-6), ("fp64", 1e-12)])
def test_prepared_runs_match_execute_batch_for_new_values(nl, oracle_mod, prec, eps):
    series = _ragged(11)
    offsets, t, dy = _layout(series)
    f0, df, nf = _grids(series)
    plan = nl.Plan(2, 1, eps, prec)
    pb = plan.prepare_batch(offsets, f0, df, nf)
    info = pb.describe()
    assert info["launches"] >= info["classes"] >= 2 and info["bytes"] > 0
    rng = np.random.default_rng(3)
    for trial in range(3):
        yv = np.concatenate([s.y * (1 + 0.5 * trial) + rng.normal(0, 0.3, s.nd) for s in series])
        y = _dev(yv)
        P = pb.run(t, y, dy).cpu().numpy()
        Q, off = plan.execute_batch(t, y, dy, offsets, f0, df, nf)
        Q = Q.cpu().numpy()
        assert np.array_equal(off, pb.out_offsets)
        for s, o in zip(series, off):
            assert_identical(P[o:o + s.nf], Q[o:o + s.nf])
        # one series against the oracle on these values
        i = trial * 3
        s, o, a = series[i], off[i], offsets[i]
        ref = oracle_mod.periodogram(s.t, yv[a:a + s.nd], s.dy, s.f0, s.df, np.arange(s.nf))
        tol = 1e-9 if prec == "fp64" else 1e-4
        assert np.max(np.abs(P[o:o + s.nf] - ref)) <= tol
    pb.close()
    plan.close()


def test_small_budget_prepares_several_launches(nl):
    series = _ragged(12, n=10)
    offsets, t, dy = _layout(series)
    f0, df, nf = _grids(series)
    y = _dev(np.concatenate([s.y for s in series]))
    big = nl.Plan(2, 1, 1e-9, "fp64")
    small = nl.Plan(2, 1, 1e-9, "fp64", batch_workspace_bytes=2_000_000)
    a = big.prepare_batch(offsets, f0, df, nf)
    b = small.prepare_batch(offsets, f0, df, nf)
    assert b.describe()["launches"] > a.describe()["launches"]
    Pa = a.run(t, y, dy).cpu().numpy()
    Pb = b.run(t, y, dy).cpu().numpy()
    assert np.max(np.abs(Pa - Pb)) <= 1e-12
    for x in (a, b, big, small):
        x.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_graph_replays_the_batch_on_new_contents(nl, prec):
    import torch
    series = _ragged(13)
    offsets, t, dy = _layout(series)
    f0, df, nf = _grids(series)
    eps = 1e-6 if prec == "fp32" else 1e-10
    plan = nl.Plan(2, 1, eps, prec)
    pb = plan.prepare_batch(offsets, f0, df, nf, normalization="psd", fit_mean=False)
    y = _dev(np.concatenate([s.y for s in series]))
    g = pb.graph(t, y, dy)
    rng = np.random.default_rng(5)
    for _ in range(3):
        y.copy_(_dev(np.concatenate([s.y + rng.normal(0, 1, s.nd) for s in series])))
        got = g.replay()
        g.sync()
        got = got.cpu().numpy()
        ref = pb.run(t, y, dy).cpu().numpy()
        direct, _ = plan.execute_batch(t, y, dy, offsets, f0, df, nf, normalization="psd",
                                       fit_mean=False)
        direct = direct.cpu().numpy()
        scale = max(1.0, float(np.max(np.abs(direct))))
        assert_identical(got, ref)
        assert_identical(got, direct)
    torch.cuda.synchronize()
    del g
    pb.close()
    plan.close()


def test_prepared_shared_layout_and_graph(nl):
    import torch
    t, Y, dy, f0, df, nf = W.uniform_batch(seed=9, nseries=40, nd=2000, nf=24_000)
    plan = nl.Plan(2, 1, 1e-6, "fp32")
    pb = plan.prepare_shared(Y.shape[0], Y.shape[1], f0, df, nf)
    tt, dd = _dev(t), _dev(dy)
    YY = _dev(Y)
    P = pb.run(tt, YY, dd).cpu().numpy()
    Q = plan.execute_shared(tt, YY, dd, f0, df, nf).cpu().numpy()
    assert P.shape == (40, nf)
    for i in range(40):
        assert_identical(P[i], Q[i], i)
    g = pb.graph(tt, YY, dd)
    YY.mul_(-2.0).add_(1.0)           # P is invariant under y -> a y + b
    got = g.replay()
    g.sync()
    got = got.cpu().numpy()
    for i in range(40):
        assert_rerun_close(got[i], Q[i], "fp32")
    torch.cuda.synchronize()
    del g
    pb.close()
    plan.close()


@pytest.mark.parametrize("fit_mean,center,norm", [(False, True, "model"), (False, False, "psd"),
                                                   (True, True, "log")])
def test_prepared_shared_layout_variants(nl, fit_mean, center, norm):
    t, Y, dy, f0, df, nf = W.uniform_batch(seed=21, nseries=24, nd=1500, nf=9000)
    Y = Y + 0.7
    plan = nl.Plan(2, 1, 1e-10, "fp64")
    model = dict(fit_mean=fit_mean, center_data=center, normalization=norm)
    pb = plan.prepare_shared(Y.shape[0], Y.shape[1], f0, df, nf, **model)
    tt, YY, dd = _dev(t), _dev(Y), _dev(dy)
    P = pb.run(tt, YY, dd).cpu().numpy()
    Q = plan.execute_shared(tt, YY, dd, f0, df, nf, **model).cpu().numpy()
    scale = max(1.0, float(np.max(np.abs(Q))))
    for i in range(Y.shape[0]):
        assert_identical(P[i], Q[i], (i, fit_mean, center, norm))
    pb.close()
    plan.close()


def test_prepare_rejects_bad_layouts(nl):
    plan = nl.Plan(2, 1, 1e-6, "fp32")
    with pytest.raises(nl.LSError):
        plan.prepare_batch([0, 1, 10], [0.1, 0.1], [0.01, 0.01], [100, 100])   # 1-point series
    with pytest.raises(nl.LSError):
        plan.prepare_batch([0, 5, 10], [0.1, 0.1], [0.01, -0.01], [100, 100])  # df <= 0
    with pytest.raises(nl.LSError):
        plan.prepare_batch([0, 5, 10], [0.1, 0.1], [0.01, 0.01], [100, 100], eps=1e-3 * 1e-6)
    plan.close()


def test_closing_the_plan_first_leaves_inert_batches(nl):
    import torch
    series = _ragged(14, n=4)
    offsets, t, dy = _layout(series)
    f0, df, nf = _grids(series)
    y = _dev(np.concatenate([s.y for s in series]))
    plan = nl.Plan(2, 1, 1e-6, "fp32")
    pb = plan.prepare_batch(offsets, f0, df, nf)
    g = pb.graph(t, y, dy)
    g.replay()
    g.sync()
    plan.close()                      # closes the batch first
    with pytest.raises(RuntimeError):
        pb.run(t, y, dy)
    with pytest.raises(RuntimeError):
        g.replay()
    pb.close()
    # the same through the C-ABI alone: the plan destroyed before its batch
    h = nl.ls_plan(2, 1, 1e-6, nl.LS_FP32)
    offs = np.ascontiguousarray(offsets)
    f0a, dfa = np.array(f0), np.array(df)
    nfa = np.array(nf, dtype=np.int64)
    oo = np.concatenate([[0], np.cumsum(nfa)[:-1]]).astype(np.int64)
    b = nl.ls_batch_prepare(h, len(series), offs.ctypes.data, f0a.ctypes.data, dfa.ctypes.data,
                            nfa.ctypes.data, oo.ctypes.data, 1e-6, 0)
    assert nl.ls_destroy(h) == 0
    out = torch.empty(int(nfa.sum()), dtype=torch.float64, device="cuda:0")
    assert nl.ls_batch_run(b, t.data_ptr(), y.data_ptr(), dy.data_ptr(), out.data_ptr()) == 1
    assert nl.ls_batch_destroy(b) == 0


def test_objects_left_alive_at_exit_tear_down_cleanly(nl, tmp_path):
    # plan, batch and graph still referenced from the main module (and from
    # functions defined there, a reference cycle) when the interpreter exits:
    # their finalizers then run in no particular order
    import subprocess
    import sys
    root = __import__("os").path.dirname(__import__("os").path.dirname(__file__))
    script = tmp_path / "leave_alive.py"
    script.write_text(f"""
import sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import paper_2409_08090_gb300 as nl
from paper_2409_08090_gb300 import workloads as W
series = [W.random_case(i, 300, 900) for i in range(5)]
off = np.zeros(6, dtype=np.int64); off[1:] = np.cumsum([s.nd for s in series])
t, y, dy = (torch.tensor(np.concatenate([getattr(s, a) for s in series]), device="cuda:0")
            for a in ("t", "y", "dy"))
plan = nl.Plan(2, 1, 1e-6, "fp32")
pb = plan.prepare_batch(off, [s.f0 for s in series], [s.df for s in series], [900] * 5)
run = lambda: pb.run(t, y, dy)
g = pb.graph(t, y, dy)
fn = g.replay
fn(); g.sync(); run()
torch.cuda.synchronize()
print("done")
""")
    r = subprocess.run([sys.executable, str(script)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "done" in r.stdout, (r.returncode, r.stderr[-2000:])
