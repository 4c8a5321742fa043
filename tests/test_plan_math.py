"""Plan arithmetic on the host: the ES kernel's Fourier transform by the
library's Gauss-Legendre rule against adaptive quadrature, and the chosen
(w, beta, n) reaching the requested tolerance against the oracle (through a
numpy model of the same steps), all without a GPU."""
import numpy as np
import pytest

from paper_2409_08090_gb300 import workloads as W


@pytest.fixture(scope="module")
def nl():
    import paper_2409_08090_gb300 as m
    m.build.build()
    return m


@pytest.mark.parametrize("w,n", [(7, 240_000), (10, 24_000), (13, 24_000), (2, 64), (16, 100)])
def test_kernel_ft_matches_adaptive_quadrature(nl, w, n):
    # phi_hat(k) = (w/2) int_{-1}^{1} psi(z) cos(pi k w z / n) dz, psi(z) =
    # exp(beta (sqrt(1 - z^2) - 1)); integrated adaptively after z = sin(theta),
    # which makes the integrand smooth, for every mode the deconvolution uses
    # (|k| <= n/4 with upsampling 2).
    from scipy.integrate import quad
    beta = 2.30 * w if w > 4 else {2: 2.20, 3: 2.26, 4: 2.38}[w] * w
    for k in (0.0, 1.0, n / 16, n / 7, n / 4):
        f = lambda th: (np.exp(beta * (np.cos(th) - 1)) * np.cos(th)
                        * np.cos(np.pi * k * w * np.sin(th) / n))
        ref = w * quad(f, 0, np.pi / 2, limit=400, epsabs=1e-16, epsrel=1e-15)[0]
        got = nl.ls_kernel_ft(k, n, w, beta)
        assert abs(got - ref) <= 2e-14 * abs(ref), (k, got, ref)


def test_kernel_ft_is_sum_of_grid_samples(nl):
    # Poisson summation: sum_m psi((m - u) 2/w) e^{2 pi i k m / n} = e^{2 pi i k u/n} phi_hat(k)
    # up to the aliasing error of the kernel (tiny for |k| <= n/4).
    w, n = 13, 64
    beta = 2.30 * w
    u = 0.3717
    m = np.arange(int(np.ceil(u - w / 2)), int(np.floor(u + w / 2)) + 1)
    z = (m - u) * 2 / w
    psi = np.exp(beta * (np.sqrt(1 - z * z) - 1))
    for k in (0, 3, 11, 16):
        lhs = np.sum(psi * np.exp(2j * np.pi * k * m / n))
        rhs = np.exp(2j * np.pi * k * u / n) * nl.ls_kernel_ft(k, n, w, beta)
        assert abs(lhs - rhs) < 1e-11 * abs(rhs)


@pytest.mark.parametrize("eps,ups", [(1e-12, 2.0), (1e-9, 2.0), (1e-6, 2.0), (1e-9, 1.5),
                                     (1e-6, 1.5)])
def test_chosen_parameters_meet_tolerance(nl, oracle_mod, eps, ups):
    from tests.nufft_model import model_sums
    s = W.single_small()
    p = nl.ls_choose_params(s.nf, eps, 0, upsampling=ups)
    sums, YY = model_sums(s.t, s.y, s.dy, s.f0, s.df, s.nf, p["width"], p["beta"], p["n"],
                          nl.ls_kernel_ft)
    k = np.arange(s.nf)
    P_o, S_o = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, k, return_sums=True)
    # NUFFT error model: |g_k error| <~ eps * sum |h_j|  (sum w^ = 1 for C, S, C2, S2)
    err = np.max(np.abs(sums - S_o[:, :6]), axis=0)
    h1 = np.sum(np.abs(s.y - np.average(s.y, weights=1 / s.dy ** 2)) / s.dy ** 2) / np.sum(1 / s.dy ** 2)
    assert err[0] < 10 * eps * h1 and err[1] < 10 * eps * h1
    assert np.all(err[2:] < 10 * eps)
    assert abs(YY - S_o[0, 6]) < 1e-14
