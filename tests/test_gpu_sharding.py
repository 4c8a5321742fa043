"""The multi-GPU split run as sequential shards on one GPU (each shard is what
one rank would compute): frequency bands of one series concatenate to the
whole periodogram, and series shards of a ragged batch reproduce the batch."""
import numpy as np
import pytest

from paper_2409_08090_gb300 import sharding as SH
from paper_2409_08090_gb300 import workloads as W
from tests.rerun_tolerance import assert_rerun_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2409_08090_gb300 as m
    m.build.build()
    m.load_library()
    return m


@pytest.mark.parametrize("prec,eps,world", [("fp64", 1e-12, 3), ("fp32", 1e-6, 4)])
def test_frequency_bands_concatenate_to_the_whole(nl, oracle_mod, prec, eps, world):
    import torch
    dev = torch.device("cuda:0")
    s = W.random_case(61, 20000, 240_001, baseline=3000.0)
    t, y, dy = (torch.tensor(a, device=dev) for a in (s.t, s.y, s.dy))
    whole_plan = nl.Plan(s.nd, s.nf, eps, prec)
    whole = whole_plan.execute(t, y, dy, s.f0, s.df).cpu().numpy()
    whole_plan.close()
    out = np.empty(s.nf)
    for r in range(world):
        f0b, nfb, lo = SH.band_grid(s.f0, s.df, s.nf, r, world)
        plan = nl.Plan(s.nd, nfb, eps, prec)
        k_lo, band = SH.band_periodogram(plan, t, y, dy, s.f0, s.df, s.nf, r, world)
        assert k_lo == lo
        out[lo:lo + nfb] = band.cpu().numpy()
        plan.close()
    # each band is a different NUFFT (own centre, own grid): both results are
    # within the parity bar of the oracle, so compare both against it
    k = np.random.default_rng(1).choice(s.nf, 400, replace=False)
    P_o = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k)
    for P in (out, whole):
        if prec == "fp64":
            assert np.max(np.abs(P[k] - P_o)) <= 1e-9
        else:
            assert np.linalg.norm(P[k] - P_o) / np.linalg.norm(P_o) <= 1e-5


def test_series_shards_reproduce_the_batch(nl):
    import torch
    dev = torch.device("cuda:0")
    series = [W.ragged_series(700 + i, nd_lo=100, nd_hi=5000) for i in range(12)]
    cost = SH.series_cost([s.nd for s in series], [s.nf for s in series])

    def run(idx):
        sub = [series[i] for i in idx]
        off = np.zeros(len(sub) + 1, dtype=np.int64)
        off[1:] = np.cumsum([s.nd for s in sub])
        cat = [torch.tensor(np.concatenate([getattr(s, a) for s in sub]), device=dev)
               for a in ("t", "y", "dy")]
        plan = nl.Plan(2, 1, 1e-9, "fp64")
        P, o = plan.execute_batch(*cat, off, [s.f0 for s in sub], [s.df for s in sub],
                                  [s.nf for s in sub])
        P = P.cpu().numpy()
        plan.close()
        return {i: P[oo:oo + series[i].nf] for i, oo in zip(idx, o)}

    whole = run(list(range(len(series))))
    for world in (2, 5):
        merged = {}
        for part in SH.series_shards(cost, world):
            if part:
                merged.update(run(part))
        for i in range(len(series)):
            assert_rerun_close(merged[i], whole[i], "fp64")
