"""Pins for the oracle's model variants: the fit_mean, center_data and
normalization options of the Astropy Lomb-Scargle interface that nifty-ls backs
(Sec. 1 of arXiv 2409.08090).  Each variant is checked against an independent
weighted least-squares fit (numpy.linalg.lstsq) and, where one exists, against
a classical closed form (the Schuster periodogram via numpy.fft).

Definitions in least-squares terms, with chi2 using the unnormalised weights
w = 1/dy^2 and chi2_ref the residual of the model without its sinusoid:
  standard 1 - chi2/chi2_ref, model chi2_ref/chi2 - 1, log ln(chi2_ref/chi2),
  psd (chi2_ref - chi2)/2.
"""
import itertools

import numpy as np
import pytest

from paper_2409_08090_gb300 import workloads as W

NORMS = ("standard", "model", "log", "psd")


def _lstsq(t, y, dy, f, fit_mean, center, norm):
    w = np.ones_like(t) if dy is None else 1.0 / np.asarray(dy) ** 2
    yc = y - np.sum(w * y) / np.sum(w) if (center or fit_mean) else y.copy()
    cols = [np.cos(2 * np.pi * f * t), np.sin(2 * np.pi * f * t)]
    if fit_mean:
        cols.append(np.ones_like(t))
    X = np.stack(cols, 1)
    sw = np.sqrt(w)
    beta, *_ = np.linalg.lstsq(X * sw[:, None], yc * sw, rcond=None)
    chi2 = np.sum(w * (yc - X @ beta) ** 2)
    chi2_ref = np.sum(w * yc ** 2)
    return {"standard": 1.0 - chi2 / chi2_ref, "model": chi2_ref / chi2 - 1.0,
            "log": np.log(chi2_ref / chi2), "psd": 0.5 * (chi2_ref - chi2)}[norm]


@pytest.mark.parametrize("fit_mean,center", [(True, True), (False, True), (False, False)])
def test_variants_equal_weighted_least_squares(oracle_mod, fit_mean, center):
    s = W.random_case(31, 400, 3000)
    y = s.y + 0.7                     # a mean that the uncentred model must carry
    rng = np.random.default_rng(4)
    k = np.sort(rng.choice(s.nf, 60, replace=False)).astype(np.int64)
    for norm in NORMS:
        P = oracle_mod.periodogram(s.t, y, s.dy, s.f0, s.df, k, fit_mean=fit_mean,
                                   center_data=center, normalization=norm)
        ref = np.array([_lstsq(s.t, y, s.dy, s.f0 + kk * s.df, fit_mean, center, norm)
                        for kk in k])
        scale = max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(P - ref)) <= 1e-10 * scale, norm


def test_fit_mean_forces_centering(oracle_mod):
    # a fitted offset absorbs the mean, so center_data has no effect with fit_mean
    s = W.random_case(32, 300, 1000)
    k = np.arange(200, dtype=np.int64)
    a = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k, center_data=True)
    b = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k, center_data=False)
    assert np.array_equal(a, b)


def test_uncentred_model_sees_the_offset(oracle_mod):
    # Without centring and without a fitted offset, adding a constant changes P;
    # with centring it does not.
    s = W.random_case(33, 300, 1000)
    k = np.arange(300, dtype=np.int64)
    kw = dict(fit_mean=False)
    P0 = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k, center_data=False, **kw)
    P1 = oracle_mod.periodogram(s.t, s.y + 3.0, s.dy, s.f0, s.df, k, center_data=False, **kw)
    assert np.max(np.abs(P0 - P1)) > 1e-3
    C0 = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k, center_data=True, **kw)
    C1 = oracle_mod.periodogram(s.t, s.y + 3.0, s.dy, s.f0, s.df, k, center_data=True, **kw)
    assert np.max(np.abs(C0 - C1)) < 1e-12


def test_pure_sinusoid_without_offset_has_unit_power(oracle_mod):
    # y = A sin(2 pi f* t + phi) exactly: the offset-free model fits it with
    # chi2 = 0 at f* = f0 + k* df, uncentred.
    rng = np.random.default_rng(8)
    t = np.sort(rng.uniform(0, 50, 500))
    dy = np.exp(rng.normal(0, 0.3, 500))
    f0, df, kstar = 0.02, 0.004, 77
    y = 2.5 * np.sin(2 * np.pi * (f0 + kstar * df) * t + 0.3)
    P = oracle_mod.periodogram(t, y, dy, f0, df, np.array([kstar - 5, kstar], dtype=np.int64),
                               fit_mean=False, center_data=False)
    assert abs(P[1] - 1.0) < 1e-12 and P[0] < 0.99


def test_psd_is_the_schuster_periodogram_for_uniform_sampling(oracle_mod):
    # t_j = j, unit weights, Fourier frequencies m/N (m != 0, 2m != 0 mod N):
    # C2 = S2 = 0, so tau = 0, CC = SS = 1/2 and the psd power is |F[m]|^2 / N of
    # the centred data (classical periodogram), with or without the fitted mean.
    N = 200
    rng = np.random.default_rng(12)
    t = np.arange(N, dtype=np.float64)
    y = rng.normal(0, 1, N) + 0.8 * np.sin(2 * np.pi * 23 * t / N) + 4.0
    F = np.fft.fft(y - y.mean())
    m = np.array([1, 9, 23, 60, 99], dtype=np.int64)
    for fit_mean in (True, False):
        P = oracle_mod.periodogram(t, y, None, 1.0 / N, 1.0 / N, m - 1, fit_mean=fit_mean,
                                   normalization="psd")
        assert np.max(np.abs(P - np.abs(F[m]) ** 2 / N)) < 1e-10


def test_normalisations_are_monotone_maps_of_each_other(oracle_mod):
    # For a fixed model, model = s/(1-s) and log = -ln(1-s) of standard s, and
    # psd = s * chi2_ref / 2: checks the normalisation branch selection.
    s = W.random_case(34, 250, 800)
    k = np.arange(400, dtype=np.int64)
    for fit_mean, center in itertools.product((True, False), (True, False)):
        out = {n: oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k, fit_mean=fit_mean,
                                         center_data=center, normalization=n) for n in NORMS}
        st = out["standard"]
        assert np.allclose(out["model"], st / (1 - st), rtol=1e-12, atol=1e-15)
        assert np.allclose(out["log"], -np.log1p(-st), rtol=1e-12, atol=1e-15)
        w = 1.0 / s.dy ** 2 if s.dy is not None else np.ones_like(s.t)
        yc = s.y - np.sum(w * s.y) / np.sum(w) if (center or fit_mean) else s.y
        assert np.allclose(out["psd"], 0.5 * st * np.sum(w * yc ** 2), rtol=1e-12)


def test_rejects_unknown_normalisation(oracle_mod):
    t = np.linspace(0, 1, 10)
    with pytest.raises(ValueError):
        oracle_mod.periodogram(t, np.sin(t), None, 0.1, 0.1, np.arange(3), normalization="x")
    # without centring, only an all-zero series is degenerate
    P = oracle_mod.periodogram(t, np.ones(10), None, 0.1, 0.1, np.arange(3), fit_mean=False,
                               center_data=False)
    assert np.all(np.isfinite(P))
    with pytest.raises(ValueError):
        oracle_mod.periodogram(t, np.zeros(10), None, 0.1, 0.1, np.arange(3), fit_mean=False,
                               center_data=False)
