"""Oracle for the floating-mean Lomb-Scargle periodogram (nifty-ls, arXiv 2409.08090).

TEST INFRASTRUCTURE ONLY.  The direct O(N_d N_f) FP64 sums of Eq. 1 and the
standard-normalised generalised power (the definitions are written out in
``ls_oracle.c``'s header).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it.

Parity status: every output is pinned by tests that do not reuse this code
(closed forms, least squares, numpy FFT special case, brute force); see
``tests/test_oracle_pins.py``.  No function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ls_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblsoracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ls_oracle.c with gcc (-O2, OpenMP, no fast-math, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.ls_oracle_power.restype = ctypes.c_int
            lib.ls_oracle_power.argtypes = [
                ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p,
                ctypes.c_void_p, ctypes.c_void_p]
            lib.ls_oracle_power_ex.restype = ctypes.c_int
            lib.ls_oracle_power_ex.argtypes = [
                ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p,
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            lib.ls_oracle_threads.restype = ctypes.c_int
            lib.ls_oracle_threads.argtypes = []
            _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the oracle's frequency loop runs on."""
    return int(_load().ls_oracle_threads())


NORMALIZATIONS = ("standard", "model", "log", "psd")


def periodogram(t, y, dy, f0: float, df: float, k, return_sums: bool = False,
                fit_mean: bool = True, center_data: bool = True,
                normalization: str = "standard"):
    """Direct FP64 periodogram at frequencies ``f0 + k*df`` for integer array ``k``.

    ``dy`` may be None (unit errors).  ``fit_mean``, ``center_data`` and
    ``normalization`` select the model variant of the Astropy interface (the
    definitions are in ``ls_oracle.c``'s header).  Returns ``P`` (float64,
    len(k)), and with ``return_sums`` also an array (len(k), 7) of
    (Ch, Sh, C, S, C2, S2, YY).
    """
    lib = _load()
    t = np.ascontiguousarray(t, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    if t.shape != y.shape or t.ndim != 1:
        raise ValueError("t and y must be 1-D arrays of equal length")
    dyp = None
    if dy is not None:
        dy = np.ascontiguousarray(np.broadcast_to(np.asarray(dy, dtype=np.float64), t.shape))
        dyp = dy.ctypes.data
    k = np.ascontiguousarray(k, dtype=np.int64)
    P = np.empty(k.shape[0], dtype=np.float64)
    sums = np.empty((k.shape[0], 7), dtype=np.float64) if return_sums else None
    if normalization not in NORMALIZATIONS:
        raise ValueError(f"normalization must be one of {NORMALIZATIONS}")
    rc = lib.ls_oracle_power_ex(t.shape[0], t.ctypes.data, y.ctypes.data, dyp,
                                float(f0), float(df), k.shape[0], k.ctypes.data,
                                int(bool(fit_mean)), int(bool(center_data)),
                                NORMALIZATIONS.index(normalization),
                                P.ctypes.data, sums.ctypes.data if sums is not None else None)
    if rc != 0:
        raise ValueError("oracle rejected the input (N_d < 1, dy <= 0 or vanishing YY)")
    return (P, sums) if return_sums else P
