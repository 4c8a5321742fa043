"""Autotuning of a plan's upsampling, spreader tile and FFT schedule, with a
JSON cache.

Three plan options trade against each other and their best values depend on
N_d / N_f and on the device:

* the upsampling sigma in {1.5, 2}: a 25% smaller fine grid (fewer FFT and HBM
  bytes) against a wider kernel (more spread work);
* the pass-A tile width (``cols_per_block`` in {1, 2, 4, 8}: fine-grid
  columns per block, which is also the bin width of the bin sort): wider tiles
  load each point record fewer times but hold fewer blocks per SM;
* the FFT schedule (``fft_max_radix`` 16 or 8 for both sub-FFTs, or the
  plan's own per-pass choice): fewer stages and barriers against lighter
  butterflies.

``tune`` measures them on the device for a request shape in three stages
(sigma with the automatic tile and schedule; then each tile width at the best
sigma; then radix 8 and 16 at the best of those: 8 plans instead of 30) and keeps the
fastest in a JSON file keyed by (device, precision, eps, N_f, N_d rounded up
to a power of two).  A stage keeps the automatic choice unless a candidate is
strictly faster.  ``Plan(..., upsampling="tuned")`` resolves through
``tuned_options``: a cache hit costs a dictionary lookup; a miss runs the
measurement once.

The cache file is ``$LS_AUTOTUNE_CACHE`` if set, else
``~/.cache/paper_2409_08090_gb300/autotune.json``; writes go through a
temporary file and an atomic rename, so concurrent processes never read a
partial file (the last writer wins for a key both tuned).
"""
from __future__ import annotations

import json
import math
import os
import threading

__all__ = ["CANDIDATES", "TILES", "RADICES", "cache_path", "cache_key", "load_cache", "tune",
           "tuned_options"]

CANDIDATES = (1.5, 2.0)        # upsampling
TILES = (1, 2, 4, 8)           # cols_per_block (0: the plan's own choice)
RADICES = (8, 16)              # fft_max_radix (0: the plan's own per-pass choice)
_lock = threading.Lock()


def cache_path() -> str:
    env = os.environ.get("LS_AUTOTUNE_CACHE")
    if env:
        return env
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2409_08090_gb300",
                        "autotune.json")


def _nd_bucket(nd: int) -> int:
    return 1 << max(1, math.ceil(math.log2(max(int(nd), 2))))


def cache_key(device_name: str, precision: str, eps: float, nf: int, nd: int) -> str:
    return f"{device_name}|{precision}|{float(eps):.3g}|{int(nf)}|{_nd_bucket(nd)}"


def config_key(cfg: dict) -> str:
    return f"s{cfg['upsampling']:g}/c{cfg['cols_per_block']}/r{cfg['fft_max_radix']}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def _save_cache(data: dict, path: str) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}.{threading.get_ident()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _device_name(device: int) -> str:
    import torch
    return torch.cuda.get_device_name(device)


def _measure_on_device(nf: int, eps: float, precision: str, nd: int, device: int,
                       reps: int):
    """Returns measure(cfg) -> median ms of one ls_execute on a synthetic series
    of the request's shape (coordinates covering a fifth of the period, like a
    long observing span at the default frequency spacing) with the plan options
    in cfg."""
    import numpy as np
    import torch

    import paper_2409_08090_gb300 as nl
    rng = np.random.default_rng(20240912)
    df = 1.0 / 5000.0
    t = np.sort(rng.uniform(0.0, 0.2 / df, nd))
    y = np.sin(2 * np.pi * 0.37 * t) + rng.normal(0.0, 0.5, nd)
    dev = torch.device("cuda", device)
    tt, yy = torch.tensor(t, device=dev), torch.tensor(y, device=dev)
    out = torch.empty(nf, dtype=torch.float64, device=dev)

    def measure(cfg: dict) -> float:
        plan = nl.Plan(nd, nf, eps, precision, device=device, upsampling=cfg["upsampling"],
                       cols_per_block=cfg["cols_per_block"],
                       fft_max_radix=cfg["fft_max_radix"])
        try:
            for _ in range(2):
                plan.execute(tt, yy, None, df, df, out=out, sync=False)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(reps)]
            for a, b in ev:
                a.record()
                plan.execute(tt, yy, None, df, df, out=out, sync=False)
                b.record()
            torch.cuda.synchronize(dev)
            nl._check(nl.ls_sync(plan.handle), "autotune measurement")
            ms = sorted(a.elapsed_time(b) for a, b in ev)
            return ms[len(ms) // 2]
        finally:
            plan.close()

    return measure


def tune(nf: int, eps: float, precision: str = "fp32", nd: int | None = None, device: int = 0,
         reps: int = 5, path: str | None = None, measure=None, device_name: str | None = None,
         force: bool = False) -> dict:
    """Measure the candidate plan options for (nf, eps, precision, nd) in three
    stages and cache the fastest.  ``measure(cfg) -> ms`` may be supplied
    (tests), cfg = {"upsampling", "cols_per_block", "fft_max_radix"}; a
    candidate the library rejects for this shape is skipped.  Returns the cache
    entry {"upsampling", "cols_per_block", "fft_max_radix", "ms": {config: ms}}."""
    nd = int(nd if nd is not None else max(2, nf // 12))
    path = path or cache_path()
    name = device_name or _device_name(device)
    key = cache_key(name, precision, eps, nf, nd)
    with _lock:
        if not force:
            hit = load_cache(path).get(key)
            if hit is not None:
                return _complete(hit)
        if measure is None:
            measure = _measure_on_device(int(nf), float(eps), precision, _nd_bucket(nd),
                                         device, reps)
        times = {}

        def run(cfg):
            try:
                ms = float(measure(dict(cfg)))
            except Exception:       # the library has no plan for these options here
                return None
            times[config_key(cfg)] = ms
            return ms

        # stage 1: the upsampling, with the plan's own tile and schedule
        best, best_ms = None, None
        for sigma in CANDIDATES:
            cfg = {"upsampling": sigma, "cols_per_block": 0, "fft_max_radix": 0}
            ms = run(cfg)
            if ms is not None and (best_ms is None or ms < best_ms):
                best, best_ms = cfg, ms
        if best is None:
            raise RuntimeError(f"no upsampling candidate could be planned for {key}")
        # stage 2: the tile width at that upsampling (strictly faster to win)
        stage = dict(best)
        for cols in TILES:
            cfg = dict(stage, cols_per_block=cols)
            ms = run(cfg)
            if ms is not None and ms < best_ms:
                best, best_ms = cfg, ms
        # stage 3: the FFT schedule
        stage = dict(best)
        for r in RADICES:
            cfg = dict(stage, fft_max_radix=r)
            ms = run(cfg)
            if ms is not None and ms < best_ms:
                best, best_ms = cfg, ms
        entry = dict(best, ms=times)
        data = load_cache(path)
        data[key] = entry
        _save_cache(data, path)
        return entry


def _complete(entry: dict) -> dict:
    """Cache entries written before the tile and schedule were tuned carry the
    upsampling only: the others are the plan's own choice."""
    out = dict(entry)
    out.setdefault("cols_per_block", 0)
    out.setdefault("fft_max_radix", 0)
    return out


def tuned_options(nf: int, eps: float, precision: str, nd: int, device: int = 0) -> dict:
    """The cached (or freshly measured) fastest plan options for this shape:
    keyword arguments of ``Plan`` (upsampling, cols_per_block, fft_max_radix)."""
    e = tune(nf, eps, precision, nd, device)
    return {"upsampling": float(e["upsampling"]), "cols_per_block": int(e["cols_per_block"]),
            "fft_max_radix": int(e["fft_max_radix"])}
