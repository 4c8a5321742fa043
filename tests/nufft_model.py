"""CPU model of the library's NUFFT arithmetic (test scaffolding only).

Re-traces, in numpy and FP64, the steps the CUDA kernels take with the
parameters the library chooses (ls_choose_params, ls_kernel_ft): pre-phase,
ES spreading onto n cells, FFT with the + sign, deconvolution by 1/phi_hat and
the power.  Used on CPU to show that the chosen (w, beta, n) meet the
tolerance against the oracle before any GPU runs, and to localise a GPU
discrepancy to a step.  It is neither the oracle nor the product.
"""
import numpy as np


def model_sums(t, y, dy, f0, df, nf, width, beta, n, kernel_ft):
    w_ = np.ones_like(t) if dy is None else 1.0 / np.asarray(dy) ** 2
    wh = w_ / w_.sum()
    ybar = np.sum(wh * y)
    yc = y - ybar
    K0 = nf // 2
    fc = f0 + K0 * df
    frac = lambda v: v - np.floor(v)
    p = np.exp(2j * np.pi * frac(fc * t))
    strengths = (wh * yc * p, wh * p, wh * p * p)
    u = (frac(df * t) * n, frac(2 * df * t) * n, )
    kp = np.arange(-K0, nf - K0)
    phat = np.array([kernel_ft(float(k), n, width, beta) for k in np.abs(kp)])
    out = []
    for s, uu in zip(strengths, (u[0], u[0], u[1])):
        G = np.zeros(n, complex)
        c0 = np.ceil(uu - width / 2).astype(np.int64)
        for i in range(width):
            m = c0 + i
            z = (m - uu) * 2 / width
            v = np.exp(beta * (np.sqrt(np.maximum(1 - z * z, 0)) - 1))
            np.add.at(G, np.mod(m, n), s * v)
        Gh = n * np.fft.ifft(G)
        out.append(Gh[np.mod(kp, n)] / phat)
    g1, g2, g3 = out
    return np.stack([g1.real, g1.imag, g2.real, g2.imag, g3.real, g3.imag], 1), np.sum(wh * yc * yc)
