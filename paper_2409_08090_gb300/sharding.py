"""Work split across GPUs, one process per GPU, with no exchange step.

The periodogram shards two ways, both embarrassingly parallel:

* a batch by series: every series is an independent problem, so each rank
  runs its share through ``Plan.execute_batch`` and the outputs are only
  concatenated;
* one large series by frequency band: the band ``[k_lo, k_hi)`` of the grid
  ``f0 + k df`` is itself the periodogram on the grid
  ``(f0 + k_lo df) + k' df, k' < k_hi - k_lo`` — an independent NUFFT with its
  own centre frequency that reads every point (the input is replicated; it is
  small next to the fine grids) and writes a disjoint slice of P.

Nothing is reduced: the only cross-rank step is the host-side gather of the
finished slices.  The split functions are pure host code (tested on CPU with
gloo ranks); ``band_periodogram`` and ``gather_bands`` are the GPU-rank
wrappers.
"""
from __future__ import annotations

import heapq

import numpy as np

__all__ = ["band_shards", "band_grid", "series_cost", "series_shards", "band_periodogram",
           "gather_bands"]


def band_shards(nf: int, world: int) -> list[tuple[int, int]]:
    """Contiguous bands [lo, hi) covering 0..nf-1, one per rank, sizes differing
    by at most one (the first nf % world bands are one longer).  Ranks beyond
    nf get empty bands."""
    if nf < 0 or world < 1:
        raise ValueError("nf >= 0 and world >= 1 required")
    base, extra = divmod(nf, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def band_grid(f0: float, df: float, nf: int, rank: int, world: int):
    """This rank's sub-grid: (f0_band, nf_band, k_lo).  f0_band = f0 + k_lo df
    is formed in FP64 like any user grid; the library treats it as exact."""
    lo, hi = band_shards(nf, world)[rank]
    return f0 + lo * df, hi - lo, lo


def series_cost(nd, nf) -> np.ndarray:
    """Relative cost of a series: its fine grids (~ nf log nf) plus its points."""
    nd = np.asarray(nd, dtype=np.float64)
    nf = np.asarray(nf, dtype=np.float64)
    return nf * np.log2(np.maximum(nf, 2.0)) + 16.0 * nd


def series_shards(costs, world: int) -> list[list[int]]:
    """Partition of series indices over ranks by longest-processing-time
    greedy assignment (largest cost first to the least-loaded rank; ties by
    rank).  Each rank's list is in increasing index order.  The heaviest rank
    carries at most the mean load plus one series' cost."""
    costs = np.asarray(costs, dtype=np.float64)
    if world < 1:
        raise ValueError("world >= 1 required")
    order = sorted(range(costs.shape[0]), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]


def band_periodogram(plan, t, y, dy, f0: float, df: float, nf: int, rank: int, world: int,
                     **model):
    """This rank's band of one series on its GPU (``plan`` sized for the band).
    Returns (k_lo, power tensor of the band); an empty band returns (k_lo, None)."""
    f0b, nfb, lo = band_grid(f0, df, nf, rank, world)
    if nfb == 0:
        return lo, None
    return lo, plan.execute(t, y, dy, f0b, df, nfb, **model)


def gather_bands(k_lo: int, band, nf: int, group=None):
    """Host-side concatenation of every rank's band (torch.distributed
    all_gather_object over the given group); returns the full float64 array
    on every rank.  ``band`` may be a tensor (any device), an array or None."""
    import torch.distributed as dist
    part = None
    if band is not None:
        part = band.detach().cpu().numpy() if hasattr(band, "detach") else np.asarray(band)
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, (int(k_lo), part), group=group)
    out = np.empty(nf, dtype=np.float64)
    seen = 0
    for lo, p in parts:
        if p is None:
            continue
        out[lo:lo + p.shape[0]] = p
        seen += p.shape[0]
    if seen != nf:
        raise RuntimeError(f"bands cover {seen} of {nf} frequencies")
    return out
