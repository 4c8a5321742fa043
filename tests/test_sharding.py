"""Multi-rank split of the periodogram (no GPU): band and series shards cover
the work exactly once, balance it, and — run as two gloo ranks that each
evaluate their share with the oracle and gather it on the host — reproduce
the single-process result bit for bit.  A band of f0 + k df is its own grid
(f0 + k_lo df) + k' df, so the oracle (exact phases) must give identical
values; series shards are independent problems."""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2409_08090_gb300 import sharding as SH
from paper_2409_08090_gb300 import workloads as W


@pytest.mark.parametrize("nf,world", [(1, 1), (10, 3), (7, 8), (12_000_000, 8), (5, 2)])
def test_band_shards_cover_the_grid_once(nf, world):
    b = SH.band_shards(nf, world)
    assert len(b) == world and b[0][0] == 0 and b[-1][1] == nf
    for (lo, hi), (lo2, _) in zip(b, b[1:]):
        assert hi == lo2
    sizes = [hi - lo for lo, hi in b]
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == nf


def test_series_shards_partition_and_balance():
    rng = np.random.default_rng(2)
    nd = np.exp(rng.uniform(np.log(100), np.log(1e5), 500)).astype(int)
    c = SH.series_cost(nd, 12 * nd)
    for world in (1, 2, 3, 8):
        parts = SH.series_shards(c, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(500))
        loads = [c[p].sum() for p in parts]
        assert max(loads) <= c.sum() / world + c.max() + 1e-6
    assert SH.series_shards([], 4) == [[], [], [], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # one series split by frequency band
        s = W.random_case(7, 300, 1001, baseline=300.0)
        f0b, nfb, lo = SH.band_grid(s.f0, s.df, s.nf, rank, world)
        band = oracle.periodogram(s.t, s.y, s.dy, f0b, s.df, np.arange(nfb)) if nfb else None
        full = SH.gather_bands(lo, band, s.nf)
        # a ragged batch split by series
        series = [W.random_case(40 + i, 50 + 37 * i, 200 + 90 * i) for i in range(7)]
        parts = SH.series_shards(SH.series_cost([x.nd for x in series], [x.nf for x in series]),
                                 world)
        mine = {i: oracle.periodogram(series[i].t, series[i].y, series[i].dy, series[i].f0,
                                      series[i].df, np.arange(series[i].nf))
                for i in parts[rank]}
        allp = [None] * world
        dist.all_gather_object(allp, mine)
        if rank == 0:
            merged = {}
            for d in allp:
                assert not set(d) & set(merged)
                merged.update(d)
            np.save(os.path.join(outdir, "band.npy"), full)
            np.savez(os.path.join(outdir, "series.npz"),
                     **{str(i): merged[i] for i in range(len(series))})
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_process_result(oracle_mod):
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True)
        full = np.load(os.path.join(d, "band.npy"))
        ser = np.load(os.path.join(d, "series.npz"))
        s = W.random_case(7, 300, 1001, baseline=300.0)
        ref = oracle_mod.periodogram(s.t, s.y, s.dy, s.f0, s.df, np.arange(s.nf))
        # the band grid f0 + lo df re-rounds f0; phases are exact, so the values
        # agree to the oracle's rounding of the phase
        assert np.max(np.abs(full - ref)) <= 1e-12
        for i in range(7):
            x = W.random_case(40 + i, 50 + 37 * i, 200 + 90 * i)
            assert np.array_equal(ser[str(i)], oracle_mod.periodogram(x.t, x.y, x.dy, x.f0, x.df,
                                                                      np.arange(x.nf)))
