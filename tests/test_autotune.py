"""Autotuner cache logic without a GPU: the fastest candidate is kept, the
cache is keyed by shape (N_d rounded up to a power of two), hits skip the
measurement, unusable candidates and damaged cache files are tolerated."""
import json

import pytest

from paper_2409_08090_gb300 import autotune as AT


def test_fastest_candidate_is_cached_and_reused(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []

    def measure(sigma):
        calls.append(sigma)
        return {1.5: 2.0, 2.0: 3.0}[sigma]

    e = AT.tune(120_000, 1e-6, "fp32", nd=10_000, path=path, measure=measure, device_name="G")
    assert e["upsampling"] == 1.5 and set(e["ms"]) == {"1.5", "2"}
    assert sorted(calls) == [1.5, 2.0]
    # same shape class (N_d 9000 rounds to the same power of two): a hit
    e2 = AT.tune(120_000, 1e-6, "fp32", nd=9_000, path=path, measure=measure, device_name="G")
    assert e2 == e and len(calls) == 2
    data = json.load(open(path))
    assert AT.cache_key("G", "fp32", 1e-6, 120_000, 10_000) in data
    # another device name or precision is a different key
    AT.tune(120_000, 1e-6, "fp64", nd=10_000, path=path, measure=lambda s: 1.0, device_name="G")
    AT.tune(120_000, 1e-6, "fp32", nd=10_000, path=path, measure=lambda s: 1.0, device_name="H")
    assert len(json.load(open(path))) == 3


def test_force_remeasures_and_ties_prefer_the_smaller_sigma(tmp_path):
    path = str(tmp_path / "c.json")
    AT.tune(5000, 1e-9, "fp64", nd=400, path=path, measure=lambda s: 1.0, device_name="G")
    e = AT.tune(5000, 1e-9, "fp64", nd=400, path=path, measure=lambda s: {1.5: 5.0, 2.0: 1.0}[s],
                device_name="G", force=True)
    assert e["upsampling"] == 2.0


def test_unplannable_candidates_are_skipped(tmp_path):
    path = str(tmp_path / "c.json")

    def measure(sigma):
        if sigma == 1.5:
            raise RuntimeError("no plan")
        return 4.0

    assert AT.tune(1000, 1e-6, "fp32", nd=100, path=path, measure=measure,
                   device_name="G")["upsampling"] == 2.0
    with pytest.raises(RuntimeError):
        AT.tune(2000, 1e-6, "fp32", nd=100, path=path,
                measure=lambda s: (_ for _ in ()).throw(RuntimeError("x")), device_name="G")


def test_damaged_cache_file_is_replaced(tmp_path):
    path = tmp_path / "c.json"
    path.write_text("{not json")
    e = AT.tune(1000, 1e-6, "fp32", nd=100, path=str(path), measure=lambda s: s,
                device_name="G")
    assert e["upsampling"] == 1.5
    assert json.loads(path.read_text())


def test_cache_path_follows_the_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("LS_AUTOTUNE_CACHE", str(tmp_path / "x.json"))
    assert AT.cache_path() == str(tmp_path / "x.json")
