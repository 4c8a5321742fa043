"""Agreement expected between two GPU evaluations of the same periodogram that
differ only in grouping (batch vs alone, served vs direct): the spread adds
with shared-memory atomics, so the summation order, and with it the last bits
of every sum, changes from run to run.  FP64: rounding level.  FP32: the sums'
rounding (~1e-7) is amplified by 1/lambda_min of the normal matrix at the
lowest frequencies, so the bound is the FP32 parity bar (max 1e-4, relative
l2 1e-5 over the whole grid)."""
import numpy as np


def assert_rerun_close(a, b, prec, scale=1.0, what=""):
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.abs(a - b)
    if prec == "fp64":
        assert np.max(d) <= 1e-12 * scale, what
    else:
        assert np.max(d) <= 1e-4 * scale, what
        assert np.linalg.norm(a - b) <= 1e-5 * max(np.linalg.norm(b), 1e-300), what
