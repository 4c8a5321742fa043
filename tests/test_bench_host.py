"""bench.py's host-side contract, without a GPU: the reference arm's JSON line
(the oracle timed on the host cores), the digest rule that keeps recorded DRAM
traffic from being reported for changed kernels, and the algorithmic-byte model
the roofline divides by."""
import importlib.util
import json
import os
import subprocess
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "single_small", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "periodograms/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["gpu_launches"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 \
        and e2e["d2h_bytes_per_step"] == 0
    # the small grid fits one step: every frequency of the grid is evaluated
    assert "12000 seeded random frequencies" in cb["sample"]


def test_recorded_traffic_requires_the_same_kernel_sources(bench, tmp_path, monkeypatch):
    fake = tmp_path / "repo"
    (fake / "paper_2409_08090_gb300" / "csrc").mkdir(parents=True)
    (fake / "profiles").mkdir()
    src = fake / "paper_2409_08090_gb300" / "csrc" / "k.cu"
    src.write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(fake))
    digest = bench.source_digest()
    (fake / "profiles" / "traffic.json").write_text(json.dumps({
        "k_passA:fp32:single_large": {"source_digest": digest, "dram_bytes_per_launch": 123}}))
    assert bench.recorded_traffic("k_passA", "fp32", "single_large") == 123
    # another workload, precision or kernel has no record
    assert bench.recorded_traffic("k_passA", "fp32", "single_medium") is None
    assert bench.recorded_traffic("k_passA", "fp64", "single_large") is None
    assert bench.recorded_traffic("k_passB", "fp32", "single_large") is None
    # any change of the kernel sources retires the record
    src.write_text("__global__ void k() { }\n")
    assert bench.source_digest() != digest
    assert bench.recorded_traffic("k_passA", "fp32", "single_large") is None


def test_committed_traffic_record_is_reported_only_for_its_sources(bench):
    # each record's total is its read + write bytes; the bench reports it only
    # while the kernel sources hash to the digest it was taken on (a kernel
    # edit retires it until the next ncu capture)
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    digest = bench.source_digest()
    for key, ent in d.items():
        if key.startswith("_"):
            continue
        assert ent["dram_bytes_per_launch"] == ent["read"] + ent["write"], key
        kernel, prec, workload = key.split(":")
        got = bench.recorded_traffic(kernel, prec, workload)
        if ent["source_digest"] == digest:
            assert got == ent["dram_bytes_per_launch"], key
        else:
            assert got is None, key


def test_algorithmic_bytes_model(bench):
    info = types.SimpleNamespace(n=18_874_368)
    nd, nf = 1_000_000, 12_000_000
    b32 = bench.algorithmic_bytes(info, nd, nf, "fp32")
    # pass A: H written once (3 n complex64) + the sorted records (cell, offset,
    # strength) of three transforms
    assert b32["pass_a_spread_fft"] == 3 * info.n * 8 + 3 * nd * (4 + 4 + 8)
    # pass B: H read once, P written, one deconvolution factor per output
    assert b32["pass_b_fft_deconv_power"] == 3 * info.n * 8 + 8 * nf + 4 * nf
    b64 = bench.algorithmic_bytes(info, nd, nf, "fp64")
    assert b64["pass_a_spread_fft"] == 3 * info.n * 16 + 3 * nd * (4 + 8 + 16)
    assert b64["pass_b_fft_deconv_power"] == 3 * info.n * 16 + 8 * nf + 8 * nf
    # the benchmark workload's figures quoted in the profiles
    assert round(b32["pass_a_spread_fft"] / 1e6, 1) == 501.0
    assert round(b32["pass_b_fft_deconv_power"] / 1e6, 1) == 597.0


def test_measured_peak_is_read_from_the_peaks_file(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm_peak() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6791.4}))
    assert bench.measured_hbm_peak() == (6791.4, "measured")
