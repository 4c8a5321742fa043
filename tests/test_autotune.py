"""Autotuner cache and search logic without a GPU: the fastest configuration is
kept, the search runs in three stages (upsampling, tile width, FFT schedule),
the cache is keyed by shape (N_d rounded up to a power of two), hits skip the
measurement, unusable candidates and damaged cache files are tolerated."""
import json

import pytest

from paper_2409_08090_gb300 import autotune as AT


def _by_sigma(table):
    return lambda cfg: table[cfg["upsampling"]]


def test_fastest_candidate_is_cached_and_reused(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []

    def measure(cfg):
        calls.append(AT.config_key(cfg))
        return {1.5: 2.0, 2.0: 3.0}[cfg["upsampling"]]

    e = AT.tune(120_000, 1e-6, "fp32", nd=10_000, path=path, measure=measure, device_name="G")
    assert e["upsampling"] == 1.5
    # ties with the automatic tile and schedule keep them
    assert e["cols_per_block"] == 0 and e["fft_max_radix"] == 0
    # 2 upsamplings + 4 tile widths + 2 schedules, each configuration once
    assert len(calls) == 8 and len(set(calls)) == 8 and set(e["ms"]) == set(calls)
    # same shape class (N_d 9000 rounds to the same power of two): a hit
    e2 = AT.tune(120_000, 1e-6, "fp32", nd=9_000, path=path, measure=measure, device_name="G")
    assert e2 == e and len(calls) == 8
    data = json.load(open(path))
    assert AT.cache_key("G", "fp32", 1e-6, 120_000, 10_000) in data
    # another device name or precision is a different key
    AT.tune(120_000, 1e-6, "fp64", nd=10_000, path=path, measure=lambda c: 1.0, device_name="G")
    AT.tune(120_000, 1e-6, "fp32", nd=10_000, path=path, measure=lambda c: 1.0, device_name="H")
    assert len(json.load(open(path))) == 3


def test_stages_pick_tile_and_schedule(tmp_path):
    path = str(tmp_path / "c.json")
    seen = []

    def measure(cfg):
        seen.append(dict(cfg))
        ms = {1.5: 10.0, 2.0: 12.0}[cfg["upsampling"]]
        ms -= {0: 0.0, 1: -1.0, 2: 0.5, 4: 1.5, 8: 1.0}[cfg["cols_per_block"]]
        ms -= 0.25 if cfg["fft_max_radix"] == 8 else 0.0
        return ms

    e = AT.tune(50_000, 1e-6, "fp32", nd=4_000, path=path, measure=measure, device_name="G")
    assert (e["upsampling"], e["cols_per_block"], e["fft_max_radix"]) == (1.5, 4, 8)
    # stage 2 runs at the stage-1 upsampling, stage 3 at the stage-2 tile
    assert all(c["upsampling"] == 1.5 for c in seen[2:])
    assert seen[-2:] == [{"upsampling": 1.5, "cols_per_block": 4, "fft_max_radix": r}
                         for r in (8, 16)]
    assert e["ms"]["s1.5/c4/r8"] == pytest.approx(8.25)


def test_force_remeasures_and_ties_prefer_the_smaller_sigma(tmp_path):
    path = str(tmp_path / "c.json")
    AT.tune(5000, 1e-9, "fp64", nd=400, path=path, measure=lambda c: 1.0, device_name="G")
    e = AT.tune(5000, 1e-9, "fp64", nd=400, path=path, measure=_by_sigma({1.5: 5.0, 2.0: 1.0}),
                device_name="G", force=True)
    assert e["upsampling"] == 2.0
    e = AT.tune(6000, 1e-9, "fp64", nd=400, path=path, measure=lambda c: 1.0, device_name="G")
    assert e["upsampling"] == 1.5


def test_unplannable_candidates_are_skipped(tmp_path):
    path = str(tmp_path / "c.json")

    def measure(cfg):
        if cfg["upsampling"] == 1.5 or cfg["cols_per_block"] == 8:
            raise RuntimeError("no plan")
        return 4.0 - (cfg["cols_per_block"] == 2)

    e = AT.tune(1000, 1e-6, "fp32", nd=100, path=path, measure=measure, device_name="G")
    assert (e["upsampling"], e["cols_per_block"]) == (2.0, 2)
    assert "s2/c8/r0" not in e["ms"]
    with pytest.raises(RuntimeError):
        AT.tune(2000, 1e-6, "fp32", nd=100, path=path,
                measure=lambda c: (_ for _ in ()).throw(RuntimeError("x")), device_name="G")


def test_damaged_cache_file_is_replaced(tmp_path):
    path = tmp_path / "c.json"
    path.write_text("{not json")
    e = AT.tune(1000, 1e-6, "fp32", nd=100, path=str(path),
                measure=lambda c: c["upsampling"], device_name="G")
    assert e["upsampling"] == 1.5
    assert json.loads(path.read_text())


def test_entries_without_tile_fields_read_as_automatic(tmp_path):
    path = tmp_path / "c.json"
    key = AT.cache_key("G", "fp32", 1e-6, 3000, 250)
    path.write_text(json.dumps({key: {"upsampling": 2.0, "ms": {"2": 1.0}}}))
    e = AT.tune(3000, 1e-6, "fp32", nd=250, path=str(path),
                measure=lambda c: pytest.fail("a cache hit must not measure"), device_name="G")
    assert (e["upsampling"], e["cols_per_block"], e["fft_max_radix"]) == (2.0, 0, 0)


def test_cache_path_follows_the_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("LS_AUTOTUNE_CACHE", str(tmp_path / "x.json"))
    assert AT.cache_path() == str(tmp_path / "x.json")
