"""Seeded synthetic time series shaped like the nifty-ls workloads (arXiv 2409.08090).

The paper times "a double-precision time series with N_d in [1e2, 1e6]" and the
Astropy default grid N_f ~ 12 N_d (Sec. 2) but ships no data; these generators
stand in for it.  This module holds no periodogram arithmetic: it only draws
inputs (numpy PCG64, FP64) that both the CUDA path and the oracle consume.

Seeds: ``20240912 + config_index`` unless given; per-series streams come from
``numpy.random.SeedSequence(seed).spawn``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20240912


@dataclass
class Series:
    """One periodogram request: data plus its frequency grid f_k = f0 + k df."""
    t: np.ndarray
    y: np.ndarray
    dy: np.ndarray | None
    f0: float
    df: float
    nf: int
    eps: float = 1e-12
    meta: dict = field(default_factory=dict)

    @property
    def nd(self) -> int:
        return int(self.t.shape[0])


def single_small(seed: int | None = None, nd: int = 1000, nf: int = 12_000) -> Series:
    """Single FP64 series: N_d times uniform in [0, 100) days (sorted),
    y = sin(2 pi 0.37 t) + N(0, 0.5^2), dy = 0.5, f0 = 0.01, df = 0.002."""
    rng = np.random.default_rng(BASE_SEED + 0 if seed is None else seed)
    t = np.sort(rng.uniform(0.0, 100.0, nd))
    y = np.sin(2 * np.pi * 0.37 * t) + rng.normal(0.0, 0.5, nd)
    dy = np.full(nd, 0.5)
    return Series(t, y, dy, 0.01, 0.002, nf, 1e-12, {"name": "single_small"})


def single_large(seed: int | None = None, nd: int = 1_000_000, nf: int = 12_000_000,
                 sort: bool = True) -> Series:
    """Large single series over a 10-year baseline [0, 3650) days with a 120-day
    seasonal gap every 365 days (days with t mod 365 in [245, 365) carry no data);
    y = three sinusoids (periods 0.5, 3.7, 41 d; amplitudes 1, 0.3, 0.1; random
    phases) + N(0, dy^2), dy ~ LogNormal(log 0.1, 0.5); f0 = 1/3650,
    df = 1/(5*3650)."""
    rng = np.random.default_rng(BASE_SEED + 1 if seed is None else seed)
    years, season = 10, 245.0
    u = rng.uniform(0.0, years * season, nd)
    t = np.floor(u / season) * 365.0 + np.mod(u, season)
    if sort:
        t = np.sort(t)
    periods = np.array([0.5, 3.7, 41.0])
    amps = np.array([1.0, 0.3, 0.1])
    phases = rng.uniform(0.0, 2 * np.pi, 3)
    dy = np.exp(rng.normal(np.log(0.1), 0.5, nd))
    y = np.zeros(nd)
    for p, a, ph in zip(periods, amps, phases):
        y += a * np.sin(2 * np.pi * t / p + ph)
    y += rng.normal(0.0, 1.0, nd) * dy
    T = 3650.0
    return Series(t, y, dy, 1.0 / T, 1.0 / (5.0 * T), nf, 1e-9,
                  {"name": "single_large", "periods": periods.tolist()})


def uniform_batch(seed: int | None = None, nseries: int = 4096, nd: int = 10_000,
                  nf: int = 120_000):
    """Batch sharing one time array: t ~ U[0, 1000) (sorted); each series
    y_s = sin(2 pi t / P_s + phi_s) + N(0, 1), P_s log-uniform in [0.1, 100] d;
    dy = 1; f0 = 1e-3, df = 1e-4.  Returns (t, Y[nseries, nd], dy, f0, df, nf)."""
    ss = np.random.SeedSequence(BASE_SEED + 2 if seed is None else seed)
    rng = np.random.default_rng(ss)
    t = np.sort(rng.uniform(0.0, 1000.0, nd))
    P = np.exp(rng.uniform(np.log(0.1), np.log(100.0), nseries))
    phi = rng.uniform(0.0, 2 * np.pi, nseries)
    Y = np.sin(2 * np.pi * t[None, :] / P[:, None] + phi[:, None])
    Y += rng.normal(0.0, 1.0, (nseries, nd))
    return t, Y, np.ones(nd), 1e-3, 1e-4, nf


def ragged_series(seed: int, nd_lo: int = 100, nd_hi: int = 100_000) -> Series:
    """One series of the ragged mix: N_d log-uniform in [nd_lo, nd_hi]; baseline
    T log-uniform in [10, 3650] d with Poisson(3) gaps of length U(0, 0.1 T);
    dy ~ LogNormal(log 0.2, 0.7); y = one sinusoid + N(0, dy^2); N_f = 12 N_d,
    df = 1/(5T), f0 = df."""
    rng = np.random.default_rng(seed)
    nd = int(round(np.exp(rng.uniform(np.log(nd_lo), np.log(nd_hi)))))
    T = float(np.exp(rng.uniform(np.log(10.0), np.log(3650.0))))
    ngaps = rng.poisson(3)
    gaps = [(s, s + rng.uniform(0.0, 0.1 * T)) for s in rng.uniform(0.0, T, ngaps)]
    t = np.empty(0)
    while t.shape[0] < nd:
        cand = rng.uniform(0.0, T, 2 * nd)
        keep = np.ones(cand.shape[0], dtype=bool)
        for a, b in gaps:
            keep &= ~((cand >= a) & (cand < b))
        t = np.concatenate([t, cand[keep]])
    t = np.sort(t[:nd])
    dy = np.exp(rng.normal(np.log(0.2), 0.7, nd))
    period = float(np.exp(rng.uniform(np.log(0.1), np.log(0.5 * T))))
    y = np.sin(2 * np.pi * t / period + rng.uniform(0, 2 * np.pi)) + rng.normal(0.0, 1.0, nd) * dy
    df = 1.0 / (5.0 * T)
    return Series(t, y, dy, df, df, 12 * nd, 1e-6, {"name": "ragged", "period": period, "T": T})


def ragged_batch(seed: int | None = None, nseries: int = 10_000,
                 nd_lo: int = 100, nd_hi: int = 100_000) -> list[Series]:
    """The ragged mix: ``nseries`` independent series drawn by ``ragged_series``."""
    ss = np.random.SeedSequence(BASE_SEED + 3 if seed is None else seed)
    seeds = [int(c.generate_state(1)[0]) for c in ss.spawn(nseries)]
    return [ragged_series(s, nd_lo, nd_hi) for s in seeds]


def poisson_arrivals(rate_hz: float, n: int, seed: int | None = None) -> np.ndarray:
    """Arrival times (s) of a Poisson stream at ``rate_hz`` requests/s."""
    rng = np.random.default_rng(BASE_SEED + 4 if seed is None else seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, n))


def random_case(seed: int, nd: int, nf: int, *, baseline: float = 50.0,
                sort: bool = True, unit_dy: bool = False, df_t: float = 0.2,
                f0_bins: float = 3.0) -> Series:
    """Small randomised case for parity tests: N_d points over ``baseline`` days,
    a sinusoid plus heteroscedastic noise, df chosen so that df * baseline =
    ``df_t`` and f0 = ``f0_bins`` * df."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(0.0, baseline, nd)
    if sort:
        t = np.sort(t)
    dy = None if unit_dy else np.exp(rng.normal(np.log(0.3), 0.4, nd))
    period = float(np.exp(rng.uniform(np.log(0.05 * baseline), np.log(0.5 * baseline))))
    noise = rng.normal(0.0, 1.0, nd) * (1.0 if dy is None else dy)
    y = 0.7 * np.sin(2 * np.pi * t / period + rng.uniform(0, 2 * np.pi)) + noise + 3.0
    df = df_t / baseline
    return Series(t, y, dy, f0_bins * df, df, nf, 1e-12, {"name": "random", "seed": seed})
