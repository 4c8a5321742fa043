"""Agreement expected between two GPU evaluations of the same periodogram.

The spread rounds every contribution to a fixed-point grid and adds the
integers exactly (order-free), so two evaluations with the same grid, tile
width and FFT schedule on the same data are bit-identical however they are
grouped (batch or alone, served or direct, graph replay or call, any
thread): ``assert_identical``.  Evaluations that differ in configuration (tile
width, FFT schedule, a frequency band's own grid) or see algebraically
equivalent data (y -> a y + b) round differently: ``assert_rerun_close``.
FP64: rounding level.  FP32: the sums' rounding (~1e-7) is amplified by
1/lambda_min of the normal matrix at the lowest frequencies, so the bound is
the FP32 parity bar (max 1e-4, relative l2 1e-5 over the whole grid)."""
import numpy as np


def assert_identical(a, b, what=""):
    a = np.asarray(a)
    b = np.asarray(b)
    assert a.shape == b.shape, what
    assert np.array_equal(a, b), (what, float(np.max(np.abs(a - b))), int(np.count_nonzero(a != b)))


def assert_rerun_close(a, b, prec, scale=1.0, what=""):
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.abs(a - b)
    if prec == "fp64":
        assert np.max(d) <= 1e-12 * scale, what
    else:
        assert np.max(d) <= 1e-4 * scale, what
        assert np.linalg.norm(a - b) <= 1e-5 * max(np.linalg.norm(b), 1e-300), what
