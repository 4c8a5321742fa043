"""Autotuning of the plan's upsampling factor, with a JSON cache.

The library picks the upsampling sigma in {2, 1.5} from a cost model (grid
cells against kernel work, ``ls_choose_params``).  The two choices trade a 25%
smaller fine grid (fewer FFT and HBM bytes) against a wider kernel (more spread
work), and which wins depends on N_d / N_f and on the device, so ``tune``
measures both on the device for a request shape and keeps the faster one in a
JSON file keyed by (device, precision, eps, N_f, N_d rounded up to a power of
two).  ``Plan(..., upsampling="tuned")`` resolves through ``tuned_upsampling``:
a cache hit costs a dictionary lookup; a miss runs the measurement once.

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

__all__ = ["CANDIDATES", "cache_path", "cache_key", "load_cache", "tune", "tuned_upsampling"]

CANDIDATES = (1.5, 2.0)
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
    """Returns measure(sigma) -> median ms of one ls_execute on a synthetic
    series of the request's shape (coordinates covering a fifth of the period,
    like a survey baseline at the default frequency spacing)."""
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

    def measure(sigma: float) -> float:
        plan = nl.Plan(nd, nf, eps, precision, device=device, upsampling=sigma)
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
    """Measure every candidate upsampling for (nf, eps, precision, nd) and cache
    the fastest.  ``measure(sigma) -> ms`` may be supplied (tests); a candidate
    the library rejects for this shape is skipped.  Returns the cache entry
    {"upsampling": sigma, "ms": {sigma: ms}}."""
    nd = int(nd if nd is not None else max(2, nf // 12))
    path = path or cache_path()
    name = device_name or _device_name(device)
    key = cache_key(name, precision, eps, nf, nd)
    with _lock:
        if not force:
            hit = load_cache(path).get(key)
            if hit is not None:
                return hit
        if measure is None:
            measure = _measure_on_device(int(nf), float(eps), precision, _nd_bucket(nd),
                                         device, reps)
        times = {}
        for sigma in CANDIDATES:
            try:
                times[sigma] = float(measure(sigma))
            except Exception:       # the library has no plan for this sigma here
                continue
        if not times:
            raise RuntimeError(f"no upsampling candidate could be planned for {key}")
        best = min(times, key=lambda s: (times[s], s))
        entry = {"upsampling": best, "ms": {f"{s:g}": v for s, v in times.items()}}
        data = load_cache(path)
        data[key] = entry
        _save_cache(data, path)
        return entry


def tuned_upsampling(nf: int, eps: float, precision: str, nd: int, device: int = 0) -> float:
    """The cached (or freshly measured) fastest upsampling for this shape."""
    return float(tune(nf, eps, precision, nd, device)["upsampling"])
