"""Model variants on the GPU (fit_mean, center_data, normalisation): every
combination against the oracle on the same seeded inputs, through the single,
ragged-batch and shared-times entry points.  The standard-normalisation
tolerances carry over through each normalisation's derivative: model
P/(1-P) has slope 1/(1-P)^2, log -ln(1-P) slope 1/(1-P), psd a constant
factor sum w (y')^2 / 2."""
import itertools

import numpy as np
import pytest

from paper_2409_08090_gb300 import workloads as W
from tests.rerun_tolerance import assert_identical

pytestmark = pytest.mark.gpu

NORMS = ("standard", "model", "log", "psd")
MODELS = [(True, True), (False, True), (False, False)]


@pytest.fixture(scope="module")
def nl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2409_08090_gb300 as m
    m.build.build()
    m.load_library()
    return m


def _slope(norm, Pstd, s, fit_mean, center):
    if norm == "model":
        return 1.0 / (1.0 - Pstd) ** 2
    if norm == "log":
        return 1.0 / (1.0 - Pstd)
    if norm == "psd":
        w = np.ones_like(s.t) if s.dy is None else 1.0 / s.dy ** 2
        yc = s.y - np.sum(w * s.y) / np.sum(w) if (center or fit_mean) else s.y
        return np.full_like(Pstd, 0.5 * np.sum(w * yc ** 2))
    return np.ones_like(Pstd)


def _check(P, ref, Pstd, s, prec, norm, fit_mean, center):
    slope = _slope(norm, Pstd, s, fit_mean, center)
    assert np.all(np.isfinite(P))
    if prec == "fp64":
        assert np.max(np.abs(P - ref) / slope) <= 1e-9, norm
    else:
        assert np.max(np.abs(P - ref) / slope) <= 1e-4, norm
        assert np.linalg.norm(P - ref) / np.linalg.norm(ref) <= 2e-5, norm


def _dev(a):
    import torch
    return None if a is None else torch.tensor(a, device="cuda:0")


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
@pytest.mark.parametrize("fit_mean,center", MODELS)
def test_single_series_variants_match_oracle(nl, oracle_mod, prec, eps, fit_mean, center):
    s = W.random_case(71, 3000, 9001, df_t=0.9, baseline=200.0)
    y = s.y + 1.3          # an offset the uncentred model must carry
    k = np.arange(s.nf)
    Pstd = oracle_mod.periodogram(s.t, y, s.dy, s.f0, s.df, k, fit_mean=fit_mean,
                                  center_data=center)
    sd = W.Series(s.t, y, s.dy, s.f0, s.df, s.nf)
    plan = nl.Plan(s.nd, s.nf, eps, prec)
    for norm in NORMS:
        ref = oracle_mod.periodogram(s.t, y, s.dy, s.f0, s.df, k, fit_mean=fit_mean,
                                     center_data=center, normalization=norm)
        P = plan.execute(_dev(s.t), _dev(y), _dev(s.dy), s.f0, s.df, normalization=norm,
                         fit_mean=fit_mean, center_data=center).cpu().numpy()
        _check(P, ref, Pstd, sd, prec, norm, fit_mean, center)
    plan.close()


def test_no_fit_mean_sums_skip_the_offset_transform(nl, oracle_mod):
    import torch
    s = W.random_case(72, 800, 3000)
    plan = nl.Plan(s.nd, s.nf, 1e-12, "fp64")
    sums = torch.empty((s.nf, 6), dtype=torch.float64, device="cuda:0")
    plan.execute(_dev(s.t), _dev(s.y), _dev(s.dy), s.f0, s.df, sums=sums, fit_mean=False,
                 center_data=False)
    got = sums.cpu().numpy()
    plan.close()
    _, ref = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, np.arange(s.nf),
                                    return_sums=True, fit_mean=False, center_data=False)
    assert np.all(got[:, 2:4] == 0.0)
    # Ch, Sh of the uncentred y, and C2, S2: within the NUFFT tolerance (sum |h| scale)
    w = np.ones_like(s.t) if s.dy is None else 1.0 / s.dy ** 2
    h1 = np.sum(w * np.abs(s.y)) / np.sum(w)
    assert np.max(np.abs(got[:, 0:2] - ref[:, 0:2])) <= 1e-10 * h1
    assert np.max(np.abs(got[:, 4:6] - ref[:, 4:6])) <= 1e-10


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_batch_variants_match_single_series(nl, prec, eps):
    import torch
    series = [W.random_case(80 + i, nd, nf, unit_dy=(i % 2 == 0))
              for i, (nd, nf) in enumerate([(300, 2000), (1200, 7001), (50, 40), (2500, 9000)])]
    offsets = np.zeros(len(series) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([s.nd for s in series])
    t = _dev(np.concatenate([s.t for s in series]))
    y = _dev(np.concatenate([s.y + 0.5 for s in series]))
    dy = _dev(np.concatenate([np.ones(s.nd) if s.dy is None else s.dy for s in series]))
    bplan = nl.Plan(2, 1, eps, prec)
    for (fit_mean, center), norm in itertools.product(MODELS, ("standard", "psd")):
        model = dict(normalization=norm, fit_mean=fit_mean, center_data=center)
        P, off = bplan.execute_batch(t, y, dy, offsets, [s.f0 for s in series],
                                     [s.df for s in series], [s.nf for s in series], **model)
        P = P.cpu().numpy()
        for s, o, a in zip(series, off, offsets[:-1]):
            plan = nl.Plan(s.nd, s.nf, eps, prec)
            P1 = plan.execute(t[a:a + s.nd].contiguous(), y[a:a + s.nd].contiguous(),
                              dy[a:a + s.nd].contiguous(), s.f0, s.df, **model).cpu().numpy()
            plan.close()
            assert_identical(P[o:o + s.nf], P1, (fit_mean, center, norm))
    bplan.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_grouped_class_variants_match_single_series(nl, oracle_mod, prec, eps):
    # many series of one grid class (different N_d, N_f, f0, df): the launches
    # that take several series per block iteration, every model variant
    import torch
    cases = [(300 + 60 * i, (280, 300, 310)[i % 3]) for i in range(9)]
    series = [W.random_case(400 + i, nd, nf, unit_dy=(i % 2 == 0), f0_bins=1.0 + 2.5 * i,
                            df_t=(0.2, 0.7)[i % 2]) for i, (nd, nf) in enumerate(cases)]
    pcode = nl.LS_FP64 if prec == "fp64" else nl.LS_FP32
    keys = [tuple(nl.ls_choose_params(s.nf, eps, pcode, max_nd=s.nd)[k] for k in ("n", "n1", "width"))
            for s in series]
    assert max(keys.count(k) for k in set(keys)) >= 6
    offsets = np.zeros(len(series) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([s.nd for s in series])
    t = _dev(np.concatenate([s.t for s in series]))
    y = _dev(np.concatenate([s.y - 0.3 for s in series]))
    dy = _dev(np.concatenate([np.ones(s.nd) if s.dy is None else s.dy for s in series]))
    bplan = nl.Plan(2, 1, eps, prec)
    for (fit_mean, center), norm in itertools.product(MODELS, ("standard", "log")):
        model = dict(normalization=norm, fit_mean=fit_mean, center_data=center)
        P, off = bplan.execute_batch(t, y, dy, offsets, [s.f0 for s in series],
                                     [s.df for s in series], [s.nf for s in series], **model)
        P = P.cpu().numpy()
        for i, (s, o, a) in enumerate(zip(series, off, offsets[:-1])):
            plan = nl.Plan(s.nd, s.nf, eps, prec)
            P1 = plan.execute(t[a:a + s.nd].contiguous(), y[a:a + s.nd].contiguous(),
                              dy[a:a + s.nd].contiguous(), s.f0, s.df, **model).cpu().numpy()
            plan.close()
            assert_identical(P[o:o + s.nf], P1, (i, fit_mean, center, norm))
        if (fit_mean, center, norm) == (False, False, "standard"):
            s, o = series[4], off[4]
            ref = oracle_mod.periodogram(s.t, s.y - 0.3, s.dy, s.f0, s.df, np.arange(s.nf),
                                         fit_mean=False, center_data=False)
            tol = 1e-9 if prec == "fp64" else 1e-4
            assert np.max(np.abs(P[o:o + s.nf] - ref)) <= tol
    bplan.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("fit_mean,center", MODELS)
def test_shared_times_variants_match_oracle(nl, oracle_mod, fit_mean, center):
    import torch
    t, Y, dy, f0, df, nf = W.uniform_batch(seed=5, nseries=12, nd=1500, nf=9000)
    Y = Y + 0.8
    plan = nl.Plan(2, 1, 1e-12, "fp64")
    P = plan.execute_shared(torch.tensor(t, device="cuda:0"), torch.tensor(Y, device="cuda:0"),
                            torch.tensor(dy, device="cuda:0"), f0, df, nf, fit_mean=fit_mean,
                            center_data=center, normalization="model").cpu().numpy()
    plan.close()
    k = np.arange(nf)
    for i in (0, 5, 11):
        s = W.Series(t, Y[i], dy, f0, df, nf)
        Pstd = oracle_mod.periodogram(t, Y[i], dy, f0, df, k, fit_mean=fit_mean,
                                      center_data=center)
        ref = oracle_mod.periodogram(t, Y[i], dy, f0, df, k, fit_mean=fit_mean,
                                     center_data=center, normalization="model")
        _check(P[i], ref, Pstd, s, "fp64", "model", fit_mean, center)


def test_unknown_model_bits_are_rejected(nl):
    s = W.random_case(90, 100, 200)
    plan = nl.Plan(s.nd, s.nf, 1e-9, "fp64")
    t, y, out = _dev(s.t), _dev(s.y), _dev(np.zeros(s.nf))
    for word in (4, 0x400, 0xFF):
        st = nl.ls_execute(plan.handle, t.data_ptr(), y.data_ptr(), None, s.nd, s.f0, s.df,
                           s.nf, 1e-9, word, out.data_ptr())
        assert st == nl.LS_ERR_UNSUPPORTED
    plan.close()


@pytest.mark.parametrize("beta", [2.3 * 7, 2.3 * 10, 2.3 * 13, 0.976 * 3.14159 * (1 - 1 / 3) * 12])
def test_double_float_kernel_evaluation_matches_fp64(nl, beta):
    # the FP64 path spreads with a double-float evaluation of psi (exp and sqrt
    # on the FP32 units) for tolerances down to 1e-11; on the kernel's peak
    # scale it must agree with the FP64 exp/sqrt evaluation to a small fraction
    # of that (x = beta (s - 1) carries about beta 2^-48)
    import ctypes
    err = ctypes.c_double()
    st = nl._lib.ls_selftest_kernel_eval(beta, 200_001, 0, ctypes.byref(err))
    assert st == nl.LS_OK
    assert err.value <= beta * 2.0 ** -48 * 1.5, err.value


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_log_normalisation_keeps_relative_accuracy_at_small_power(nl, oracle_mod, prec, eps):
    # -ln(1 - P) ~ P for small P: where P < 1e-5 the log-normalised output must
    # carry no more relative error than the standard power itself (forming
    # 1 - P in FP32 first loses everything below P ~ 6e-8).
    s = W.random_case(91, 2000, 20000, df_t=0.9, baseline=300.0)
    k = np.arange(s.nf)
    ref_std = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k)
    ref_log = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k, normalization="log")
    plan = nl.Plan(s.nd, s.nf, eps, prec)
    P_std = plan.execute(_dev(s.t), _dev(s.y), _dev(s.dy), s.f0, s.df).cpu().numpy()
    P_log = plan.execute(_dev(s.t), _dev(s.y), _dev(s.dy), s.f0, s.df,
                         normalization="log").cpu().numpy()
    plan.close()
    small = ref_std < 1e-5
    assert np.count_nonzero(small) >= 50
    rel_std = np.abs(P_std[small] / ref_std[small] - 1.0)
    rel_log = np.abs(P_log[small] / ref_log[small] - 1.0)
    bound = 3.0 * float(np.max(rel_std)) + 1e-6
    assert float(np.max(rel_log)) <= bound, (float(np.max(rel_log)), bound)
    if prec == "fp64":
        assert float(np.max(rel_log)) <= 1e-5


def test_double_assembly_matches_fp64_add(nl):
    # the FP32 path writes its double-float power as a double assembled on the
    # integer pipe: bit for bit the FP64 conversions and add, on 2^24 generated
    # pairs including powers of two, ties and non-finite values
    import ctypes
    bad = ctypes.c_int64(-1)
    st = nl._lib.ls_selftest_double_assembly(1 << 24, 20240914, 0, ctypes.byref(bad))
    assert st == 0 and bad.value == 0, (st, bad.value)
