"""GB300-native Lomb-Scargle periodograms via type-1 NUFFT (method of nifty-ls,
arXiv 2409.08090).

The compute path is the CUDA library ``libnifty_ls.so`` (``csrc/``, C-ABI in
``include/nifty_ls.h``).  This module is a thin ctypes binding with the same
entry-point names (``ls_plan``, ``ls_execute``, ...) plus a small convenience
layer (``Plan``, ``lombscargle``) that marshals torch tensors or numpy arrays.
Every step of the periodogram runs in the library's kernels; there is no CPU
fallback: if the library is missing, calls raise ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref

from . import build as _build

__all__ = ["LSError", "Plan", "GraphedExecute", "lombscargle", "load_library", "LS_FP64", "LS_FP32",
           "LS_NORM_STANDARD", "LS_NORM_MODEL", "LS_NORM_LOG", "LS_NORM_PSD",
           "LS_NO_FIT_MEAN", "LS_NO_CENTER", "NORMALIZATIONS", "mode_word", "ls_plan", "ls_execute", "ls_execute_sums", "ls_sync",
           "ls_destroy", "ls_set_stream", "ls_execute_noalloc", "ls_execute_batch", "ls_execute_batch_shared", "ls_plan_describe", "ls_status_str",
           "ls_choose_params", "ls_kernel_ft", "PlanInfo", "PlanOpts", "ls_timing_enable",
           "ls_timing_report", "STAGE_NAMES", "PreparedBatch", "GraphedBatch", "ls_batch_prepare",
           "ls_batch_prepare_shared", "ls_batch_run", "ls_batch_describe", "ls_batch_destroy",
           "ls_kernel_launches"]

LS_FP64, LS_FP32 = 0, 1
LS_NORM_STANDARD, LS_NORM_MODEL, LS_NORM_LOG, LS_NORM_PSD = range(4)
LS_NO_FIT_MEAN, LS_NO_CENTER = 0x100, 0x200
NORMALIZATIONS = ("standard", "model", "log", "psd")
LS_OK, LS_ERR_ARG, LS_ERR_NOMEM, LS_ERR_CUDA, LS_ERR_TIMEOUT, LS_ERR_DEGENERATE, \
    LS_ERR_UNSUPPORTED = range(7)

_c_void_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double


class PlanInfo(ctypes.Structure):
    _fields_ = [("nf", _i64), ("max_nd", _i64), ("n", _i64), ("n1", _i32), ("n2", _i32),
                ("width", _i32), ("prec", _i32), ("beta", _dbl), ("eps", _dbl),
                ("sigma", _dbl), ("workspace_bytes", _i64), ("cols_per_block", _i32),
                ("fft_max_radix", _i32), ("batch_bytes", _i64)]


class LSError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        msg = ls_status_str(status)
        super().__init__(f"{where}: {msg} (status {status})" if where else msg)


_lib = None
_lock = threading.Lock()

_SIGS = {
    "ls_plan": (ctypes.c_int, [ctypes.POINTER(_c_void_p), _i64, _i64, _dbl, ctypes.c_int,
                               ctypes.c_int, _c_void_p]),
    "ls_set_stream": (ctypes.c_int, [_c_void_p, _c_void_p]),
    "ls_execute": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i64, _dbl, _dbl,
                                  _i64, _dbl, ctypes.c_int, _c_void_p]),
    "ls_execute_sums": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i64, _dbl,
                                       _dbl, _i64, _dbl, ctypes.c_int, _c_void_p, _c_void_p]),
    "ls_sync": (ctypes.c_int, [_c_void_p]),
    "ls_plan_describe": (ctypes.c_int, [_c_void_p, ctypes.POINTER(PlanInfo)]),
    "ls_plan_reserve_batch": (ctypes.c_int, [_c_void_p]),
    "ls_destroy": (ctypes.c_int, [_c_void_p]),
    "ls_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "ls_choose_params": (ctypes.c_int, [_i64, _dbl, ctypes.c_int, _i64, _dbl,
                                        ctypes.POINTER(_i32), ctypes.POINTER(_dbl),
                                        ctypes.POINTER(_i64), ctypes.POINTER(_i32),
                                        ctypes.POINTER(_i32), ctypes.POINTER(_dbl)]),
    "ls_plan_ex": (ctypes.c_int, [ctypes.POINTER(_c_void_p), _i64, _i64, _dbl, ctypes.c_int,
                                  ctypes.c_int, _c_void_p, ctypes.c_void_p]),
    "ls_kernel_ft": (_dbl, [_dbl, _i64, _i32, _dbl]),
    "ls_selftest_double_assembly": (ctypes.c_int, [_i64, ctypes.c_uint64, ctypes.c_int,
                                                   ctypes.POINTER(_i64)]),
    "ls_selftest_kernel_eval": (ctypes.c_int, [_dbl, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(_dbl)]),
    "ls_execute_batch": (ctypes.c_int, [_c_void_p, _i64, _c_void_p, _c_void_p, _c_void_p,
                                        _c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_void_p,
                                        _dbl, ctypes.c_int, _c_void_p]),
    "ls_execute_batch_shared": (ctypes.c_int, [_c_void_p, _i64, _i64, _c_void_p, _c_void_p,
                                               _c_void_p, _dbl, _dbl, _i64, _dbl, ctypes.c_int,
                                               _c_void_p]),
    "ls_execute_noalloc": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _i64, _dbl, _dbl,
                                          _i64, _dbl, ctypes.c_int, _c_void_p, _c_void_p]),
    "ls_batch_prepare": (ctypes.c_int, [_c_void_p, ctypes.POINTER(_c_void_p), _i64, _c_void_p,
                                        _c_void_p, _c_void_p, _c_void_p, _c_void_p, _dbl,
                                        ctypes.c_int]),
    "ls_batch_prepare_shared": (ctypes.c_int, [_c_void_p, ctypes.POINTER(_c_void_p), _i64, _i64,
                                               _dbl, _dbl, _i64, _dbl, ctypes.c_int]),
    "ls_batch_run": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_void_p]),
    "ls_batch_describe": (ctypes.c_int, [_c_void_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                         ctypes.POINTER(_i64)]),
    "ls_batch_destroy": (ctypes.c_int, [_c_void_p]),
    "ls_kernel_launches": (ctypes.c_int, [ctypes.POINTER(_i64)]),
    "ls_timing_enable": (ctypes.c_int, [_c_void_p, ctypes.c_int]),
    "ls_timing_report": (ctypes.c_int, [_c_void_p, ctypes.POINTER(_dbl), ctypes.POINTER(_i64)]),
}

LS_NUM_STAGES = 4
STAGE_NAMES = ("preprocess", "bin_sort", "pass_a_spread_fft", "pass_b_fft_deconv_power")


def load_library(path: str | None = None):
    """Load libnifty_ls.so (built in-tree by ``build.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or _build.LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(
                f"CUDA library not built ({path} missing); run "
                "`python -m paper_2409_08090_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != LS_OK:
        raise LSError(status, where)


# ---- raw C-ABI mirrors (same names, plain integers/pointers) ----------------

def ls_status_str(status: int) -> str:
    return load_library().ls_status_str(int(status)).decode()


class PlanOpts(ctypes.Structure):
    _fields_ = [("upsampling", _dbl), ("batch_workspace_bytes", ctypes.c_uint64),
                ("cols_per_block", _i32), ("fft_max_radix", _i32)]


def ls_plan(max_nd: int, nf: int, eps: float, prec: int = LS_FP64, device: int = 0,
            stream: int = 0, upsampling: float = 0.0, batch_workspace_bytes: int = 0,
            cols_per_block: int = 0, fft_max_radix: int = 0) -> int:
    """Plan handle; ``upsampling`` 0 (automatic), 2.0 or 1.5, the batch
    workspace budget in bytes (0: automatic), the pass-A tile width in columns
    and the largest FFT radix (0: automatic), all through ls_plan_ex."""
    h = _c_void_p()
    lib = load_library()
    if upsampling or batch_workspace_bytes or cols_per_block or fft_max_radix:
        opts = PlanOpts(float(upsampling), int(batch_workspace_bytes), int(cols_per_block),
                        int(fft_max_radix))
        st = lib.ls_plan_ex(ctypes.byref(h), int(max_nd), int(nf), float(eps), int(prec),
                            int(device), _c_void_p(stream or None), ctypes.byref(opts))
    else:
        st = lib.ls_plan(ctypes.byref(h), int(max_nd), int(nf), float(eps), int(prec),
                         int(device), _c_void_p(stream or None))
    _check(st, "ls_plan")
    return h.value


def ls_set_stream(plan: int, stream: int) -> None:
    _check(load_library().ls_set_stream(_c_void_p(plan), _c_void_p(stream or None)),
           "ls_set_stream")


def ls_execute(plan: int, t: int, y: int, dy: int | None, nd: int, f0: float, df: float,
               nf: int, eps: float, norm: int, power: int) -> int:
    return load_library().ls_execute(_c_void_p(plan), _c_void_p(t), _c_void_p(y),
                                     _c_void_p(dy or None), int(nd), float(f0), float(df),
                                     int(nf), float(eps), int(norm), _c_void_p(power))


def ls_execute_sums(plan: int, t: int, y: int, dy: int | None, nd: int, f0: float, df: float,
                    nf: int, eps: float, norm: int, power: int | None, sums: int) -> int:
    return load_library().ls_execute_sums(_c_void_p(plan), _c_void_p(t), _c_void_p(y),
                                          _c_void_p(dy or None), int(nd), float(f0), float(df),
                                          int(nf), float(eps), int(norm),
                                          _c_void_p(power or None), _c_void_p(sums))


def ls_execute_noalloc(t: int, y: int, dy: int | None, nd: int, f0: float, df: float, nf: int,
                       eps: float, prec: int, power: int, stream: int = 0) -> int:
    """Periodogram of a small series on the library's fixed scratch area (no
    allocation, for callers that cannot allocate device memory); device
    pointers only; synchronous; returns the status code."""
    return load_library().ls_execute_noalloc(_c_void_p(t), _c_void_p(y), _c_void_p(dy or None),
                                             int(nd), float(f0), float(df), int(nf), float(eps),
                                             int(prec), _c_void_p(power),
                                             _c_void_p(stream or None))


def ls_execute_batch(plan: int, nseries: int, offsets: int, t: int, y: int, dy: int | None,
                     f0: int, df: int, nf: int, out_offsets: int, eps: float, norm: int,
                     power: int) -> int:
    """Raw C-ABI call; offsets, f0, df, nf, out_offsets are host addresses."""
    return load_library().ls_execute_batch(_c_void_p(plan), int(nseries), _c_void_p(offsets),
                                           _c_void_p(t), _c_void_p(y), _c_void_p(dy or None),
                                           _c_void_p(f0), _c_void_p(df), _c_void_p(nf),
                                           _c_void_p(out_offsets), float(eps), int(norm),
                                           _c_void_p(power))


def ls_execute_batch_shared(plan: int, nseries: int, nd: int, t: int, Y: int, dy: int | None,
                            f0: float, df: float, nf: int, eps: float, norm: int,
                            power: int) -> int:
    return load_library().ls_execute_batch_shared(_c_void_p(plan), int(nseries), int(nd),
                                                  _c_void_p(t), _c_void_p(Y),
                                                  _c_void_p(dy or None), float(f0), float(df),
                                                  int(nf), float(eps), int(norm), _c_void_p(power))


def ls_sync(plan: int) -> int:
    return load_library().ls_sync(_c_void_p(plan))


def ls_destroy(plan: int) -> int:
    return load_library().ls_destroy(_c_void_p(plan))


def ls_plan_describe(plan: int) -> PlanInfo:
    info = PlanInfo()
    _check(load_library().ls_plan_describe(_c_void_p(plan), ctypes.byref(info)),
           "ls_plan_describe")
    return info


def ls_plan_reserve_batch(plan: int) -> None:
    _check(load_library().ls_plan_reserve_batch(_c_void_p(plan)), "ls_plan_reserve_batch")


def ls_choose_params(nf: int, eps: float, prec: int = LS_FP64, max_nd: int | None = None,
                     upsampling: float = 0.0) -> dict:
    w, b, n, n1, n2, sg = _i32(), _dbl(), _i64(), _i32(), _i32(), _dbl()
    nd = max(1, int(nf) // 12) if max_nd is None else int(max_nd)
    _check(load_library().ls_choose_params(int(nf), float(eps), int(prec), nd, float(upsampling),
                                           ctypes.byref(w), ctypes.byref(b), ctypes.byref(n),
                                           ctypes.byref(n1), ctypes.byref(n2), ctypes.byref(sg)),
           "ls_choose_params")
    return {"width": w.value, "beta": b.value, "n": n.value, "n1": n1.value, "n2": n2.value,
            "sigma": sg.value}


def ls_batch_prepare(plan: int, nseries: int, offsets: int, f0: int, df: int, nf: int,
                     out_offsets: int, eps: float, norm: int) -> int:
    """Prepared-batch handle; offsets, f0, df, nf, out_offsets are host addresses."""
    h = _c_void_p()
    _check(load_library().ls_batch_prepare(_c_void_p(plan), ctypes.byref(h), int(nseries),
                                           _c_void_p(offsets), _c_void_p(f0), _c_void_p(df),
                                           _c_void_p(nf), _c_void_p(out_offsets), float(eps),
                                           int(norm)), "ls_batch_prepare")
    return h.value


def ls_batch_prepare_shared(plan: int, nseries: int, nd: int, f0: float, df: float, nf: int,
                            eps: float, norm: int) -> int:
    h = _c_void_p()
    _check(load_library().ls_batch_prepare_shared(_c_void_p(plan), ctypes.byref(h), int(nseries),
                                                  int(nd), float(f0), float(df), int(nf),
                                                  float(eps), int(norm)),
           "ls_batch_prepare_shared")
    return h.value


def ls_batch_run(batch: int, t: int, y: int, dy: int | None, power: int) -> int:
    return load_library().ls_batch_run(_c_void_p(batch), _c_void_p(t), _c_void_p(y),
                                       _c_void_p(dy or None), _c_void_p(power))


def ls_batch_describe(batch: int) -> dict:
    a, b, c = _i64(), _i64(), _i64()
    _check(load_library().ls_batch_describe(_c_void_p(batch), ctypes.byref(a), ctypes.byref(b),
                                            ctypes.byref(c)), "ls_batch_describe")
    return {"launches": a.value, "classes": b.value, "bytes": c.value}


def ls_batch_destroy(batch: int) -> int:
    return load_library().ls_batch_destroy(_c_void_p(batch))


def ls_kernel_launches() -> int:
    """Pipeline kernels enqueued through the library by this process so far."""
    c = _i64()
    _check(load_library().ls_kernel_launches(ctypes.byref(c)), "ls_kernel_launches")
    return c.value


def ls_timing_enable(plan: int, enable: bool = True) -> None:
    _check(load_library().ls_timing_enable(_c_void_p(plan), int(bool(enable))),
           "ls_timing_enable")


def ls_timing_report(plan: int) -> tuple[list, int]:
    """Summed device ms per stage (STAGE_NAMES) and the number of executes."""
    ms = (_dbl * LS_NUM_STAGES)()
    cnt = _i64()
    _check(load_library().ls_timing_report(_c_void_p(plan), ms, ctypes.byref(cnt)),
           "ls_timing_report")
    return list(ms), cnt.value


def ls_kernel_ft(k: float, n: int, width: int, beta: float) -> float:
    return float(load_library().ls_kernel_ft(float(k), int(n), int(width), float(beta)))


# ---- convenience layer ---------------------------------------------------------

def _prec_code(precision) -> int:
    if precision in (LS_FP64, "fp64", "float64", "f64", "double"):
        return LS_FP64
    if precision in (LS_FP32, "fp32", "float32", "f32", "single"):
        return LS_FP32
    raise ValueError(f"unknown precision {precision!r}")


def mode_word(normalization: str = "standard", fit_mean: bool = True,
              center_data: bool = True) -> int:
    """The ``norm`` argument of the execute calls: an ls_norm value OR'ed with
    LS_NO_FIT_MEAN / LS_NO_CENTER (the Astropy interface's options)."""
    if normalization not in NORMALIZATIONS:
        raise ValueError(f"normalization must be one of {NORMALIZATIONS}")
    word = NORMALIZATIONS.index(normalization)
    if not fit_mean:
        word |= LS_NO_FIT_MEAN
        if not center_data:
            word |= LS_NO_CENTER
    return word


class Plan:
    """Owns one ``ls_plan`` (workspace + tables for ``nf`` frequencies at ``eps``).

    Every execute method takes the model options as keywords:
    ``normalization`` ("standard", "model", "log", "psd"), ``fit_mean`` and
    ``center_data`` (see ``mode_word``)."""

    def __init__(self, max_nd: int, nf: int, eps: float = 1e-9, precision="fp64",
                 device: int = 0, upsampling: float | str = 0.0, batch_workspace_bytes: int = 0,
                 cols_per_block: int = 0, fft_max_radix: int = 0):
        """``upsampling`` 0 (the plan's cost model), 2.0 or 1.5, or "tuned":
        upsampling, tile width and FFT schedule measured per shape and cached
        (``autotune``; explicit ``cols_per_block`` / ``fft_max_radix`` are then
        ignored)."""
        self.prec = _prec_code(precision)
        self.device = int(device)
        if upsampling == "tuned":        # measured per shape, cached (autotune.py)
            from . import autotune
            opts = autotune.tuned_options(
                nf, eps, "fp32" if self.prec == LS_FP32 else "fp64", max_nd, self.device)
            upsampling = opts["upsampling"]
            cols_per_block = opts["cols_per_block"]
            fft_max_radix = opts["fft_max_radix"]
        self.handle = ls_plan(max_nd, nf, eps, self.prec, self.device, 0, upsampling,
                              batch_workspace_bytes, cols_per_block, fft_max_radix)
        self.info = ls_plan_describe(self.handle)
        self._batches = weakref.WeakSet()

    def reserve_batch(self):
        """Allocate the batch workspaces now (``ls_plan_reserve_batch``), so
        that batch calls within the plan's batch budget allocate nothing."""
        ls_plan_reserve_batch(self.handle)

    def device_bytes(self) -> int:
        """Device memory the plan holds: its single-series workspace and
        tables, its batch workspaces and its grid classes' tables."""
        info = ls_plan_describe(self.handle)
        return int(info.workspace_bytes + info.batch_bytes)

    def close(self):
        """Destroy the plan (its prepared batches first: finalizers of objects
        in a reference cycle run in no particular order)."""
        for b in list(getattr(self, "_batches", ())):
            b.close()
        if getattr(self, "handle", None):
            ls_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self) -> int:
        import torch
        return torch.cuda.current_stream(self.device).cuda_stream

    def execute(self, t, y, dy, f0: float, df: float, nf: int | None = None, eps=None,
                out=None, sums=None, sync: bool = True, **model):
        """Periodogram of one series.  ``t, y, dy`` are float64 CUDA tensors on the
        plan's device (``dy`` may be None); returns ``out`` (float64, nf)."""
        import torch
        nf = int(self.info.nf if nf is None else nf)
        eps = float(self.info.eps if eps is None else eps)
        for a in (t, y) + ((dy,) if dy is not None else ()):
            if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()):
                raise ValueError("t, y, dy must be contiguous float64 CUDA tensors")
        if out is None:
            out = torch.empty(nf, dtype=torch.float64, device=t.device)
        ls_set_stream(self.handle, self._stream())
        nd = int(t.numel())
        dyp = dy.data_ptr() if dy is not None else None
        if sums is not None:
            st = ls_execute_sums(self.handle, t.data_ptr(), y.data_ptr(), dyp, nd, f0, df, nf,
                                 eps, mode_word(**model), out.data_ptr(), sums.data_ptr())
        else:
            st = ls_execute(self.handle, t.data_ptr(), y.data_ptr(), dyp, nd, f0, df, nf, eps,
                            mode_word(**model), out.data_ptr())
        _check(st, "ls_execute")
        if sync:
            _check(ls_sync(self.handle), "ls_execute (device status)")
        return out

    def prepare_batch(self, offsets, f0, df, nf, eps=None, **model) -> "PreparedBatch":
        """Prepare the layout of a ragged batch (arguments as for
        ``execute_batch``, without the data): ``PreparedBatch.run`` then
        computes it for new values with kernels only."""
        import numpy as np
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        ns = offsets.shape[0] - 1
        f0 = np.ascontiguousarray(np.broadcast_to(np.asarray(f0, dtype=np.float64), (ns,)))
        df = np.ascontiguousarray(np.broadcast_to(np.asarray(df, dtype=np.float64), (ns,)))
        nf = np.ascontiguousarray(np.broadcast_to(np.asarray(nf, dtype=np.int64), (ns,)))
        out_off = np.zeros(ns, dtype=np.int64)
        if ns > 1:
            out_off[1:] = np.cumsum(nf)[:-1]
        eps = float(self.info.eps if eps is None else eps)
        ls_set_stream(self.handle, self._stream())
        h = ls_batch_prepare(self.handle, ns, offsets.ctypes.data, f0.ctypes.data, df.ctypes.data,
                             nf.ctypes.data, out_off.ctypes.data, eps, mode_word(**model))
        pb = PreparedBatch(self, h, (int(nf.sum()),), out_off)
        self._batches.add(pb)
        return pb

    def prepare_shared(self, nseries: int, nd: int, f0: float, df: float, nf: int, eps=None,
                       **model) -> "PreparedBatch":
        """Prepare a uniform batch (arguments as for ``execute_shared``)."""
        eps = float(self.info.eps if eps is None else eps)
        ls_set_stream(self.handle, self._stream())
        h = ls_batch_prepare_shared(self.handle, nseries, nd, f0, df, nf, eps, mode_word(**model))
        pb = PreparedBatch(self, h, (int(nseries), int(nf)), None)
        self._batches.add(pb)
        return pb

    def graph(self, t, y, dy, f0: float, df: float, nf: int | None = None, eps=None, out=None,
              **model) -> "GraphedExecute":
        """Record this execute (device buffers t, y, dy, out fixed) as a CUDA graph;
        ``.replay()`` then re-runs it on whatever the buffers hold, with one
        launch instead of one per kernel.  See ``GraphedExecute``."""
        return GraphedExecute(self, t, y, dy, f0, df, nf, eps, out, model)

    def execute_batch(self, t, y, dy, offsets, f0, df, nf, eps=None, out=None,
                      sync: bool = True, **model):
        """Periodograms of a ragged batch.  ``t, y, dy``: concatenated float64 CUDA
        tensors (``dy`` may be None); ``offsets``: nseries+1 point offsets;
        ``f0, df, nf``: per-series grids (sequences).  Returns ``(power, out_offsets)``
        with series s's power at ``power[out_offsets[s]:out_offsets[s] + nf[s]]``."""
        import numpy as np
        import torch
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        ns = offsets.shape[0] - 1
        f0 = np.ascontiguousarray(np.broadcast_to(np.asarray(f0, dtype=np.float64), (ns,)))
        df = np.ascontiguousarray(np.broadcast_to(np.asarray(df, dtype=np.float64), (ns,)))
        nf = np.ascontiguousarray(np.broadcast_to(np.asarray(nf, dtype=np.int64), (ns,)))
        out_off = np.zeros(ns, dtype=np.int64)
        if ns > 1:
            out_off[1:] = np.cumsum(nf)[:-1]
        total = int(nf.sum())
        if out is None:
            out = torch.empty(total, dtype=torch.float64, device=t.device)
        eps = float(self.info.eps if eps is None else eps)
        ls_set_stream(self.handle, self._stream())
        st = ls_execute_batch(self.handle, ns, offsets.ctypes.data, t.data_ptr(), y.data_ptr(),
                              dy.data_ptr() if dy is not None else None, f0.ctypes.data,
                              df.ctypes.data, nf.ctypes.data, out_off.ctypes.data, eps,
                              mode_word(**model), out.data_ptr())
        _check(st, "ls_execute_batch")
        if sync:
            _check(ls_sync(self.handle), "ls_execute_batch (device status)")
        return out, out_off

    def execute_shared(self, t, Y, dy, f0: float, df: float, nf: int, eps=None, out=None,
                       sync: bool = True, **model):
        """Uniform batch: series Y[s] (a 2-D float64 CUDA tensor, one row per
        series) all observed at times ``t`` with uncertainties ``dy`` (or None).
        Returns power as a (nseries, nf) tensor."""
        import torch
        ns, nd = int(Y.shape[0]), int(Y.shape[1])
        if out is None:
            out = torch.empty((ns, int(nf)), dtype=torch.float64, device=Y.device)
        eps = float(self.info.eps if eps is None else eps)
        ls_set_stream(self.handle, self._stream())
        st = ls_execute_batch_shared(self.handle, ns, nd, t.data_ptr(), Y.data_ptr(),
                                     dy.data_ptr() if dy is not None else None, f0, df, nf, eps,
                                     mode_word(**model), out.data_ptr())
        _check(st, "ls_execute_batch_shared")
        if sync:
            _check(ls_sync(self.handle), "ls_execute_batch_shared (device status)")
        return out

    def execute_host(self, t, y, dy, f0: float, df: float, nf: int | None = None, eps=None,
                     out=None, **model):
        """Same, with host (numpy float64) buffers: the library copies in and out."""
        import numpy as np
        nf = int(self.info.nf if nf is None else nf)
        eps = float(self.info.eps if eps is None else eps)
        t = np.ascontiguousarray(t, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        dyp = None
        if dy is not None:
            dy = np.ascontiguousarray(dy, dtype=np.float64)
            dyp = dy.ctypes.data
        if out is None:
            out = np.empty(nf, dtype=np.float64)
        ls_set_stream(self.handle, self._stream())
        st = ls_execute(self.handle, t.ctypes.data, y.ctypes.data, dyp, t.shape[0], f0, df, nf,
                        eps, mode_word(**model), out.ctypes.data)
        _check(st, "ls_execute")
        return out


def _record(plan: "Plan", run, device: int):
    """Warm a run up outside capture (first-use set-up of the kernels), then
    record one run as a CUDA graph.  "relaxed": the library queries pointer
    attributes while recording."""
    import torch
    side = torch.cuda.Stream(device=device)
    side.wait_stream(torch.cuda.current_stream(device))
    with torch.cuda.stream(side):
        run()
    torch.cuda.current_stream(device).wait_stream(side)
    torch.cuda.synchronize(device)
    _check(ls_sync(plan.handle), "graph warm-up (device status)")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="relaxed"):
        run()
    torch.cuda.synchronize(device)
    return graph


class GraphedExecute:
    """One ``ls_execute`` recorded by CUDA stream capture (torch.cuda.CUDAGraph).

    With device buffers, ls_execute enqueues only kernels and a memset on the
    plan's stream, so it can be captured; a replay re-runs the whole pipeline
    on the current contents of ``t, y, dy`` (same N_d, grid and model) and
    writes ``out``.  Device-side errors accumulate in the plan's status word:
    ``sync()`` waits and raises them.  The plan must outlive the graph and must
    not run other work concurrently with a replay (they share its workspace).
    """

    def __init__(self, plan: "Plan", t, y, dy, f0, df, nf, eps, out, model):
        import torch
        self.plan = plan
        nf = int(plan.info.nf if nf is None else nf)
        self.out = out if out is not None else torch.empty(nf, dtype=torch.float64,
                                                            device=t.device)
        self._args = (t, y, dy, f0, df, nf, eps)
        self.graph = _record(plan, lambda: plan.execute(t, y, dy, f0, df, nf, eps, out=self.out,
                                                         sync=False, **model), plan.device)

    def replay(self):
        """Enqueue the recorded pipeline on the current stream's device."""
        if not self.plan.handle:
            raise RuntimeError("the plan of this graph was closed: its memory is gone")
        self.graph.replay()
        return self.out

    def sync(self):
        """Wait for the replays on the current stream and raise their device
        errors.  The plan's stream is set to the current stream first: the
        plan last ran on the capture's stream, which replays are not ordered
        with, and the status read must follow the replays."""
        ls_set_stream(self.plan.handle, self.plan._stream())
        _check(ls_sync(self.plan.handle), "graph replay (device status)")
        return self.out


class PreparedBatch:
    """A batch layout prepared once (``ls_batch_prepare`` / ``_shared``).

    ``run(t, y, dy)`` computes the periodograms of new values in that layout
    (ragged: concatenated t, y, dy as for ``Plan.execute_batch``; shared: t, dy
    of nd values and Y of nseries x nd) with kernels only, and ``graph``
    records a run as a CUDA graph.  Output: ragged, a flat tensor with series
    s at ``out_offsets[s]``; shared, (nseries, nf).  The plan must outlive
    the batch; runs on one plan must not overlap."""

    def __init__(self, plan: "Plan", handle: int, shape: tuple, out_offsets):
        self.plan = plan
        self.handle = handle
        self.shape = shape
        self.out_offsets = out_offsets

    def describe(self) -> dict:
        return ls_batch_describe(self.handle)

    def _out(self, like, out):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device=like.device)
        return out

    def run(self, t, y, dy, out=None, sync: bool = True):
        import torch
        if not self.handle:
            raise RuntimeError("this prepared batch was closed")
        for a in (t, y) + ((dy,) if dy is not None else ()):
            if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()):
                raise ValueError("t, y, dy must be contiguous float64 CUDA tensors")
        out = self._out(t, out)
        ls_set_stream(self.plan.handle, self.plan._stream())
        _check(ls_batch_run(self.handle, t.data_ptr(), y.data_ptr(),
                            dy.data_ptr() if dy is not None else None, out.data_ptr()),
               "ls_batch_run")
        if sync:
            _check(ls_sync(self.plan.handle), "ls_batch_run (device status)")
        return out

    def graph(self, t, y, dy, out=None) -> "GraphedBatch":
        return GraphedBatch(self, t, y, dy, self._out(t, out))

    def close(self):
        if getattr(self, "handle", None):
            ls_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GraphedBatch:
    """One ``PreparedBatch.run`` recorded as a CUDA graph: a replay re-runs
    every launch of the batch (over the plan's batch streams) on the current
    contents of t, y, dy.  ``sync()`` raises device-side errors.  The batch
    must outlive the graph."""

    def __init__(self, batch: PreparedBatch, t, y, dy, out):
        self.batch = batch
        self.out = out
        self._args = (t, y, dy)
        self.graph = _record(batch.plan, lambda: batch.run(t, y, dy, out=out, sync=False),
                             batch.plan.device)

    def replay(self):
        if not self.batch.handle:
            raise RuntimeError("the batch of this graph was closed: its memory is gone")
        self.graph.replay()
        return self.out

    def sync(self):
        """As GraphedExecute.sync: the status is read on the current stream."""
        ls_set_stream(self.batch.plan.handle, self.batch.plan._stream())
        _check(ls_sync(self.batch.plan.handle), "graph replay (device status)")
        return self.out


_plan_cache: dict = {}


def lombscargle(t, y, dy=None, *, f0: float, df: float, nf: int, eps: float = 1e-9,
                precision="fp64", device: int = 0, normalization: str = "standard",
                fit_mean: bool = True, center_data: bool = True):
    """Lomb-Scargle power at f0 + k df, k < nf (default: floating mean,
    standard normalisation; the keywords select the other variants).

    Accepts float64 CUDA tensors (result: CUDA tensor) or array-likes (result:
    numpy array, host buffers copied by the library).  Plans are cached per
    (device, nf, eps, precision) and grown when a longer series arrives.
    """
    prec = _prec_code(precision)
    try:
        import torch
        is_tensor = isinstance(t, torch.Tensor)
    except ImportError:  # pragma: no cover
        is_tensor = False
    nd = int(t.numel() if is_tensor else len(t))
    key = (device, int(nf), float(eps), prec)
    plan = _plan_cache.get(key)
    if plan is None or plan.info.max_nd < nd:
        if plan is not None:
            plan.close()
        plan = Plan(max(nd, 2), nf, eps, prec, device)
        _plan_cache[key] = plan
    model = dict(normalization=normalization, fit_mean=fit_mean, center_data=center_data)
    if is_tensor:
        return plan.execute(t, y, dy, f0, df, nf, eps, **model)
    return plan.execute_host(t, y, dy, f0, df, nf, eps, **model)
