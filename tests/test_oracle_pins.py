"""Pins for the oracle: each check comes from something other than the oracle's
own formulas (closed forms, invariances of the least-squares model, numpy FFT,
numpy least squares, brute force, arbitrary-precision phases).

The power is the generalised (floating-mean) Lomb-Scargle periodogram with
standard normalisation: P(f) = 1 - chi2_min(f) / chi2_0 of the weighted fit
y ~ a cos 2 pi f t + b sin 2 pi f t + c (VanderPlas 2018, cited in Sec. 1 of
arXiv 2409.08090); the sums are Eq. 1 of that paper.
"""
import math

import numpy as np
import pytest

from paper_2409_08090_gb300 import workloads as W


def _k_all(nf):
    return np.arange(nf, dtype=np.int64)


def test_pure_sinusoid_on_grid_frequency_has_unit_power(oracle_mod):
    # P1: noise-free sinusoid plus offset at f* = f0 + k* df fits exactly (chi2 = 0).
    rng = np.random.default_rng(1)
    t = np.sort(rng.uniform(0, 100, 1000))
    dy = np.exp(rng.normal(0, 0.3, 1000))
    kstar = 180
    fstar = 0.01 + kstar * 0.002
    y = 1.7 * np.sin(2 * np.pi * fstar * t + 0.4) + 5.0
    k = np.array([kstar - 3, kstar, kstar + 7], dtype=np.int64)
    P = oracle_mod.periodogram(t, y, dy, 0.01, 0.002, k)
    assert abs(P[1] - 1.0) < 1e-12
    assert P[0] < 1.0 - 1e-3 and P[2] < 1.0 - 1e-3


def test_power_is_bounded(oracle_mod):
    # P2: a ratio of explained to total weighted variance lies in [0, 1].
    for seed in range(4):
        s = W.random_case(seed, 300, 2000, unit_dy=(seed % 2 == 0))
        P = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, _k_all(s.nf))
        assert np.all(P >= -1e-14) and np.all(P <= 1 + 1e-12)


def test_invariances(oracle_mod):
    # P3: the fit is unchanged by a time shift (phase absorbed by a, b), an affine
    # map of y (absorbed by the offset and the scale of chi2) and a common scale of dy.
    s = W.random_case(11, 400, 3000)
    k = _k_all(s.nf)
    P = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k)
    P_shift = oracle_mod.periodogram(s.t + 123.456, s.y, s.dy, s.f0, s.df, k)
    P_affine = oracle_mod.periodogram(s.t, -3.5 * s.y + 17.0, s.dy, s.f0, s.df, k)
    P_dy = oracle_mod.periodogram(s.t, s.y, 7.0 * s.dy, s.f0, s.df, k)
    assert np.max(np.abs(P_shift - P)) < 1e-11
    assert np.max(np.abs(P_affine - P)) < 1e-12
    assert np.max(np.abs(P_dy - P)) < 1e-12


def test_aliasing_with_integer_times(oracle_mod):
    # P4: with integer t_j, f and f + 1 give identical phases, hence identical P.
    rng = np.random.default_rng(5)
    t = np.sort(rng.choice(np.arange(0, 400), 150, replace=False)).astype(np.float64)
    y = np.sin(2 * np.pi * 0.123 * t) + rng.normal(0, 0.5, t.shape[0])
    dy = np.exp(rng.normal(0, 0.2, t.shape[0]))
    k = _k_all(500)
    P = oracle_mod.periodogram(t, y, dy, 0.003, 0.0011, k)
    P1 = oracle_mod.periodogram(t, y, dy, 1.003, 0.0011, k)
    P7 = oracle_mod.periodogram(t, y, dy, 7.003, 0.0011, k)
    assert np.max(np.abs(P1 - P)) < 1e-11
    assert np.max(np.abs(P7 - P)) < 1e-11


def test_uniform_sampling_matches_numpy_fft(oracle_mod):
    # P5: t_j = j, equal weights, f = m/N with m != 0 and 2m != 0 mod N: the
    # mean, cos and sin columns are orthogonal, C = S = C2 = S2 = 0 and
    # P = 2 |sum y' e^{i w t}|^2 / (N sum y'^2), read off numpy.fft.fft.
    N = 256
    rng = np.random.default_rng(9)
    t = np.arange(N, dtype=np.float64)
    y = rng.normal(0, 1, N) + np.cos(2 * np.pi * 17 * t / N)
    yc = y - y.mean()
    F = np.fft.fft(yc)
    m = np.array([1, 5, 17, 40, 100, 127], dtype=np.int64)
    # frequencies f = f0 + k df with f0 = df = 1/N -> m = k + 1
    P, sums = oracle_mod.periodogram(t, y, None, 1.0 / N, 1.0 / N, m - 1, return_sums=True)
    expected = 2.0 * np.abs(F[m]) ** 2 / (N * np.sum(yc ** 2))
    assert np.max(np.abs(P - expected)) < 1e-13
    assert np.max(np.abs(sums[:, 2:6])) < 1e-13
    # Ch + i Sh = sum w^ y' e^{+i w t} = conj(F[m]) / N  (numpy's forward sign is -)
    assert np.max(np.abs(sums[:, 0] - F[m].real / N)) < 1e-13
    assert np.max(np.abs(sums[:, 1] + F[m].imag / N)) < 1e-13


def _lstsq_power(t, y, dy, f):
    w = 1.0 / dy ** 2
    sw = np.sqrt(w)
    X = np.stack([np.cos(2 * np.pi * f * t), np.sin(2 * np.pi * f * t), np.ones_like(t)], 1)
    beta, *_ = np.linalg.lstsq(X * sw[:, None], y * sw, rcond=None)
    chi2 = np.sum(w * (y - X @ beta) ** 2)
    ybar = np.sum(w * y) / np.sum(w)
    chi2_0 = np.sum(w * (y - ybar) ** 2)
    return 1.0 - chi2 / chi2_0


def test_power_equals_weighted_least_squares(oracle_mod):
    # P6: the standard-normalised generalised power is 1 - chi2_min / chi2_0 of the
    # three-parameter weighted fit, solved here by numpy.linalg.lstsq.
    s = W.random_case(21, 500, 4000)
    rng = np.random.default_rng(3)
    k = np.sort(rng.choice(s.nf, 200, replace=False)).astype(np.int64)
    P = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k)
    ref = np.array([_lstsq_power(s.t, s.y, s.dy, s.f0 + kk * s.df) for kk in k])
    assert np.max(np.abs(P - ref)) < 1e-11
    # the peak of a strong sinusoid: near-unit power also matches
    t = s.t
    y = 2.0 * np.sin(2 * np.pi * 0.2 * t + 1.0) + 0.01 * np.cos(3.3 * t)
    P = oracle_mod.periodogram(t, y, s.dy, 0.2, 1e-3, np.arange(3, dtype=np.int64))
    ref = np.array([_lstsq_power(t, y, s.dy, 0.2 + i * 1e-3) for i in range(3)])
    assert np.max(np.abs(P - ref)) < 1e-10


def test_sums_match_brute_force_loops(oracle_mod):
    # P7: tiny inputs, straight Python loops with math.sin/math.cos and no
    # phase reduction; checks every sum's sign, index and weight.
    rng = np.random.default_rng(13)
    for trial in range(20):
        nd = int(rng.integers(2, 9))
        nf = int(rng.integers(1, 17))
        t = rng.uniform(0, 10, nd)
        y = rng.normal(0, 1, nd)
        dy = rng.uniform(0.5, 2.0, nd)
        f0, df = float(rng.uniform(0, 1)), float(rng.uniform(0.01, 0.3))
        P, sums = oracle_mod.periodogram(t, y, dy, f0, df, _k_all(nf), return_sums=True)
        wts = [1.0 / (d * d) for d in dy]
        Wt = sum(wts)
        wh = [x / Wt for x in wts]
        ybar = sum(a * b for a, b in zip(wh, y))
        for i in range(nf):
            f = f0 + i * df
            row = [0.0] * 7
            for j in range(nd):
                a = 2 * math.pi * f * t[j]
                row[0] += wh[j] * (y[j] - ybar) * math.cos(a)
                row[1] += wh[j] * (y[j] - ybar) * math.sin(a)
                row[2] += wh[j] * math.cos(a)
                row[3] += wh[j] * math.sin(a)
                row[4] += wh[j] * math.cos(2 * a)
                row[5] += wh[j] * math.sin(2 * a)
                row[6] += wh[j] * (y[j] - ybar) ** 2
            assert np.max(np.abs(np.array(row) - sums[i])) < 1e-12, (trial, i)
            if nd >= 3:
                assert abs(P[i] - _lstsq_power(t, y, dy, f)) < 1e-8
            elif abs(np.exp(2j * np.pi * f * t[0]) - np.exp(2j * np.pi * f * t[1])) > 1e-3:
                # two points are fitted exactly by offset + sinusoid: chi2 = 0
                assert abs(P[i] - 1.0) < 1e-9, (trial, i)


def test_two_point_series_have_unit_power(oracle_mod):
    # Degenerate normal matrix, rank one: two points are fitted exactly by an
    # offset plus a sinusoid whenever their phasors e^{i w t_1}, e^{i w t_2}
    # differ, so chi2 = 0 and P = 1.  After the tau rotation one of CC_tau,
    # SS_tau is zero up to rounding and its term must be dropped; keeping it
    # (0/0) or dropping the other term too (a threshold above the nonzero
    # eigenvalue, ~ |e^{i w t_1} - e^{i w t_2}|^2 w^_1 w^_2) breaks P = 1.
    rng = np.random.default_rng(7)
    for trial in range(200):
        t = rng.uniform(0, 50, 2)
        y = rng.normal(0, 1, 2)
        dy = rng.uniform(0.3, 3, 2)
        f0, df = float(rng.uniform(0, 1)), float(rng.uniform(1e-3, 0.1))
        k = _k_all(64)
        f = f0 + k * df
        sep = np.abs(np.exp(2j * np.pi * f * t[0]) - np.exp(2j * np.pi * f * t[1]))
        P = oracle_mod.periodogram(t, y, dy, f0, df, k)
        m = sep > 1e-3
        assert np.all(np.isfinite(P)), trial
        assert np.max(np.abs(P[m] - 1.0)) < 1e-9, trial


def _fit_power(X, y, dy):
    # 1 - chi2_min / chi2_0 of the weighted least-squares fit on the columns X.
    w = 1.0 / dy ** 2
    sw = np.sqrt(w)
    beta, *_ = np.linalg.lstsq(X * sw[:, None], y * sw, rcond=None)
    chi2 = np.sum(w * (y - X @ beta) ** 2)
    ybar = np.sum(w * y) / np.sum(w)
    return 1.0 - chi2 / np.sum(w * (y - ybar) ** 2)


def test_collinear_phases_reduce_to_one_sinusoid(oracle_mod):
    # Times t_j = n_j + delta (n_j integers) at f = 1/2 + m: every phase is
    # delta/2 or delta/2 + 1/2 cycles, so all phasors lie on one line through the
    # origin and cos(w t), sin(w t) are both multiples of (-1)^n_j.  The model
    # then holds one sinusoid column, (-1)^n, besides the offset: the vanishing
    # eigenvalue's term must be dropped and P equals that two-column fit
    # (numpy lstsq).  The tilt delta makes the rounding of the vanishing
    # CC_tau or SS_tau land on either side of zero, so a zero threshold (keeping
    # a rounding-level denominator) fails here.
    rng = np.random.default_rng(11)
    for trial in range(100):
        n = int(rng.integers(3, 40))
        delta = float(rng.uniform(0, 1))
        tn = np.sort(rng.choice(np.arange(0, 400), n, replace=False)).astype(np.float64)
        t = tn + delta
        y = rng.normal(0, 1, n)
        dy = rng.uniform(0.3, 3, n)
        P = oracle_mod.periodogram(t, y, dy, 0.5, 1.0, _k_all(3))   # f = 1/2, 3/2, 5/2
        ref = _fit_power(np.stack([(-1.0) ** tn, np.ones(n)], 1), y, dy)
        assert np.max(np.abs(P - ref)) < 1e-12, trial


def test_integer_frequency_on_integer_times_has_zero_power(oracle_mod):
    # Integer t at integer f: every phasor is 1, cos(w t) duplicates the offset
    # column and sin(w t) vanishes, so both eigenvalues of the normal matrix are
    # zero, the sinusoid explains nothing and P = 0.
    rng = np.random.default_rng(12)
    for trial in range(20):
        n = int(rng.integers(3, 60))
        t = np.sort(rng.choice(np.arange(0, 500), n, replace=False)).astype(np.float64)
        y = rng.normal(0, 1, n)
        dy = rng.uniform(0.3, 3, n)
        P = oracle_mod.periodogram(t, y, dy, 0.0, 1.0, _k_all(4))
        assert np.max(np.abs(P)) < 1e-14, trial


def test_long_baseline_phase_reduction_is_exact(oracle_mod):
    # The phase f_k t_j of the large workload reaches ~2e6 cycles; the oracle's
    # double-double reduction must agree with 50-digit arithmetic (mpmath).
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.default_rng(17)
    t = rng.uniform(0, 3650, 6)
    y = rng.normal(0, 1, 6)
    f0, df = 1.0 / 3650, 1.0 / 18250
    k = np.array([0, 1234567, 11_999_999], dtype=np.int64)
    _, sums = oracle_mod.periodogram(t, y, None, f0, df, k, return_sums=True)
    ybar = sum(mpmath.mpf(v) for v in y) / 6
    for i, kk in enumerate(k):
        f = mpmath.mpf(f0) + int(kk) * mpmath.mpf(df)
        S = sum(mpmath.sin(2 * mpmath.pi * f * mpmath.mpf(tj)) / 6 for tj in t)
        C2 = sum(mpmath.cos(4 * mpmath.pi * f * mpmath.mpf(tj)) / 6 for tj in t)
        Ch = sum((mpmath.mpf(yj) - ybar) * mpmath.cos(2 * mpmath.pi * f * mpmath.mpf(tj)) / 6
                 for tj, yj in zip(t, y))
        assert abs(float(S) - sums[i, 3]) < 1e-14
        assert abs(float(C2) - sums[i, 4]) < 1e-14
        assert abs(float(Ch) - sums[i, 0]) < 1e-14


def test_rejects_bad_input(oracle_mod):
    t = np.linspace(0, 1, 10)
    with pytest.raises(ValueError):
        oracle_mod.periodogram(t, np.ones(10), None, 0.1, 0.1, _k_all(3))  # YY = 0
    with pytest.raises(ValueError):
        oracle_mod.periodogram(t, np.arange(10.0), np.zeros(10), 0.1, 0.1, _k_all(3))


def test_golden_regression(oracle_mod):
    # Values written by tests/golden/make_golden.py (which calls only oracle/):
    # guards the oracle against accidental drift between commits.
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "single_small_oracle.json")
    g = json.load(open(path))
    s = W.single_small()
    k = np.array(g["k"], dtype=np.int64)
    P = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k)
    assert np.max(np.abs(P - np.array(g["P"]))) < 1e-14
