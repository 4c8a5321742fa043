"""Tunable plan options on the GPU: every spreader tile width and FFT schedule
gives the same periodogram (to rounding) as the plan's own choice and stays
within the oracle tolerances, for single series and ragged batches."""
import itertools

import numpy as np
import pytest

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


def _dev(a):
    import torch
    return torch.tensor(a, device="cuda:0")


CASES = [("fp32", 1e-6, 20_000, 240_000), ("fp64", 1e-12, 3_000, 36_000)]


@pytest.mark.parametrize("prec,eps,nd,nf", CASES)
def test_tile_and_schedule_options_keep_the_result(nl, oracle_mod, prec, eps, nd, nf):
    s = W.random_case(31, nd, nf, baseline=300.0, df_t=0.2)
    t, y, dy = _dev(s.t), _dev(s.y), _dev(s.dy)
    base = nl.Plan(nd, nf, eps, prec)
    auto_cols = base.info.cols_per_block
    assert auto_cols in (1, 2, 4, 8) and base.info.fft_max_radix in (8, 16)
    P0 = base.execute(t, y, dy, s.f0, s.df).cpu().numpy()
    base.close()
    rng = np.random.default_rng(7)
    k = np.sort(rng.choice(nf, 400, replace=False))
    ref = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k)
    honoured = 0
    for cols, radix in itertools.product((1, 2, 4, 8), (0, 8, 16)):
        plan = nl.Plan(nd, nf, eps, prec, cols_per_block=cols, fft_max_radix=radix)
        info = plan.info
        assert info.cols_per_block in (cols, auto_cols)
        assert info.fft_max_radix in ((2, 4, 8, 16) if radix == 8 else (8, 16))
        honoured += info.cols_per_block == cols
        P = plan.execute(t, y, dy, s.f0, s.df).cpu().numpy()
        plan.close()
        if prec == "fp64":      # double-float FFT: rounding changes with the schedule
            assert np.max(np.abs(P - P0)) <= 1e-10, (cols, radix)
        else:
            assert_rerun_close(P, P0, prec, 1.0, (cols, radix))
        if prec == "fp64":
            assert np.max(np.abs(P[k] - ref)) <= 1e-9
        else:
            assert np.linalg.norm(P[k] - ref) / np.linalg.norm(ref) <= 1e-5
    assert honoured >= 4


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-6), ("fp64", 1e-10)])
def test_batch_classes_take_the_options(nl, prec, eps):
    import torch
    series = [W.random_case(90 + i, nd, nf) for i, (nd, nf) in
              enumerate([(300, 2000), (1200, 7001), (300, 2100), (2500, 9000), (800, 7100)])]
    offsets = np.zeros(len(series) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([s.nd for s in series])
    t = _dev(np.concatenate([s.t for s in series]))
    y = _dev(np.concatenate([s.y for s in series]))
    dy = _dev(np.concatenate([s.dy for s in series]))
    outs = []
    for cols, radix in ((0, 0), (1, 8), (4, 0), (8, 8)):
        plan = nl.Plan(2, 1, eps, prec, cols_per_block=cols, fft_max_radix=radix)
        P, off = plan.execute_batch(t, y, dy, offsets, [s.f0 for s in series],
                                    [s.df for s in series], [s.nf for s in series])
        outs.append(P.cpu().numpy())
        plan.close()
    for P in outs[1:]:
        for s, o in zip(series, off):
            if prec == "fp64":      # double-float FFT: rounding changes with the schedule
                assert np.max(np.abs(P[o:o + s.nf] - outs[0][o:o + s.nf])) <= 1e-10
            else:
                assert_rerun_close(P[o:o + s.nf], outs[0][o:o + s.nf], "fp32")
    torch.cuda.synchronize()
