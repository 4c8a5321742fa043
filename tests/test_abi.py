"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/nifty_ls.h; host-only queries return the parameters the
plan math promises."""
import ctypes
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nifty_ls.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2409_08090_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(ls_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ls_plan", "ls_execute", "ls_destroy", "ls_sync", "ls_status_str"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_model_words_match_the_header():
    import paper_2409_08090_gb300 as nl
    src = open(HEADER).read()
    for name in ("LS_NORM_STANDARD", "LS_NORM_MODEL", "LS_NORM_LOG", "LS_NORM_PSD"):
        m = re.search(name + r"\s*=\s*(\d+)", src)
        assert m and int(m.group(1)) == getattr(nl, name), name
    for name in ("LS_NO_FIT_MEAN", "LS_NO_CENTER"):
        m = re.search(r"#define\s+" + name + r"\s+(0x[0-9a-fA-F]+)", src)
        assert m and int(m.group(1), 16) == getattr(nl, name), name
    assert nl.mode_word() == 0
    assert nl.mode_word("psd", fit_mean=False, center_data=False) == 3 | 0x100 | 0x200
    # centring is implied by a fitted mean
    assert nl.mode_word("log", fit_mean=True, center_data=False) == 2
    with pytest.raises(ValueError):
        nl.mode_word("power")


def test_status_strings():
    import paper_2409_08090_gb300 as nl
    assert nl.ls_status_str(0) == "ok"
    assert "degenerate" in nl.ls_status_str(5)
    assert nl.ls_status_str(99) == "unknown status"


ODD = (1, 3, 5, 9, 15, 25, 27, 45, 75, 81, 125)


def _is_allowed(n):
    m = n
    while m % 2 == 0:
        m //= 2
    return m in ODD


@pytest.mark.parametrize("nf,eps,prec,ups,w,n", [
    (12_000, 1e-12, 0, 0.0, 13, 24_576),          # sigma 1.5 is not offered below 1e-10
    (12_000, 1e-9, 0, 2.0, 10, 24_576),
    (12_000, 1e-6, 1, 2.0, 7, 24_576),
    (12_000_000, 1e-6, 1, 2.0, 7, 25_165_824),
    (12_000_000, 1e-6, 1, 1.5, 8, 18_874_368),
    (12_000_000, 1e-9, 0, 2.0, 10, 25_165_824),
    (120_000, 1e-6, 1, 2.0, 7, 245_760),
])
def test_choose_params(nf, eps, prec, ups, w, n):
    import paper_2409_08090_gb300 as nl
    p = nl.ls_choose_params(nf, eps, prec, upsampling=ups)
    assert p["width"] == w
    assert p["n"] == n
    assert p["n1"] * p["n2"] == p["n"]
    sigma = p["sigma"]
    if sigma == 2.0:
        assert abs(p["beta"] - 2.30 * w) < 1e-12
    else:
        assert sigma == 1.5
        assert abs(p["beta"] - 0.976 * np.pi * (1 - 0.5 / sigma) * w) < 1e-12
        assert w == int(np.ceil(np.log(1 / eps) / (np.pi * np.sqrt(1 - 1 / sigma))))
    # split limits of the two passes (pass B holds three rows of N1, pass A
    # columns of N2, in shared memory); N1 a power of two
    assert 32 <= p["n1"] <= 4096
    assert p["n1"] & (p["n1"] - 1) == 0
    assert p["n2"] <= (25600 if prec == 1 else 12800) and p["n2"] % 2 == 0
    assert p["n"] >= sigma * nf


def test_automatic_upsampling_prefers_the_smaller_grid_when_fft_dominates():
    import paper_2409_08090_gb300 as nl
    big = nl.ls_choose_params(12_000_000, 1e-6, 1, max_nd=1_000_000)
    assert big["sigma"] == 1.5
    # a spread-dominated plan (many points, few frequencies) keeps sigma 2
    few = nl.ls_choose_params(1_000, 1e-6, 1, max_nd=10_000_000)
    assert few["sigma"] == 2.0


def test_choose_params_rejects():
    import paper_2409_08090_gb300 as nl
    with pytest.raises(nl.LSError):
        nl.ls_choose_params(0, 1e-6, 0)
    with pytest.raises(nl.LSError):
        nl.ls_choose_params(100, 1e-9, 1)   # FP32 cannot reach 1e-9
    with pytest.raises(nl.LSError):
        nl.ls_choose_params(100, 0.5, 0)


def test_grid_sizes_are_minimal_admissible():
    import paper_2409_08090_gb300 as nl
    for nf in (1, 2, 7, 100, 999, 4097, 65_537, 1_234_567):
        p = nl.ls_choose_params(nf, 1e-9, 0, upsampling=2.0)
        n = p["n"]
        nmin = max(2 * nf, 2 * p["width"], 64)
        assert n >= nmin and _is_allowed(n)
        # no admissible size in [nmin, n): n = c 2^k splits as N1 = 2^k1 >= 32
        # (a power of two) times an even N2, so k >= 6
        smaller = [c * 2 ** k for c in ODD for k in range(6, 40) if nmin <= c * 2 ** k < n]
        assert not smaller, (nf, n, smaller[:3])


def test_choose_params_is_cheap_enough_for_per_series_calls():
    # a ragged batch chooses parameters for every series on each call
    import time

    import paper_2409_08090_gb300 as nl
    nl.load_library()
    t0 = time.perf_counter()
    for i in range(2000):
        nl.ls_choose_params(1000 + 600 * i, 1e-6, nl.LS_FP32, 100 + 50 * i)
    assert time.perf_counter() - t0 < 2.0


def _struct_fields(name):
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", src).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            out += [v.strip() for v in decl.split(None, 1)[1].split(",")]
    return out


def test_option_and_info_structs_match_the_header():
    import paper_2409_08090_gb300 as nl
    assert [f[0] for f in nl.PlanOpts._fields_] == _struct_fields("ls_plan_opts")
    assert [f[0] for f in nl.PlanInfo._fields_] == _struct_fields("ls_plan_info")


@pytest.mark.parametrize("opt", [dict(cols_per_block=3), dict(cols_per_block=16),
                                 dict(fft_max_radix=4), dict(fft_max_radix=32),
                                 dict(upsampling=1.25)])
def test_plan_options_are_validated_before_any_device_work(opt):
    # argument checks run on the host, ahead of the device query
    import paper_2409_08090_gb300 as nl
    with pytest.raises(nl.LSError) as e:
        nl.ls_plan(1000, 12_000, 1e-6, nl.LS_FP32, **opt)
    assert e.value.status == 1


def test_prepared_batch_entry_points_reject_null_handles():
    # argument checks only: no device is touched
    import paper_2409_08090_gb300 as nl
    lib = nl.load_library()
    assert lib.ls_batch_run(None, None, None, None, None) == 1
    assert lib.ls_batch_destroy(None) == 1
    assert lib.ls_batch_describe(None, None, None, None) == 1
    h = ctypes.c_void_p(1234)
    assert lib.ls_batch_prepare(None, ctypes.byref(h), 1, None, None, None, None, None,
                                1e-6, 0) == 1
    assert h.value is None
    h = ctypes.c_void_p(1234)
    assert lib.ls_batch_prepare_shared(None, ctypes.byref(h), 4, 100, 0.1, 0.01, 1000,
                                       1e-6, 0) == 1
    assert h.value is None


@pytest.mark.parametrize("prec,eps,ups", [(1, 1e-6, 2.0), (1, 1e-6, 1.5), (0, 1e-9, 1.5),
                                          (0, 1e-12, 2.0)])
def test_grid_choice_is_minimal_for_every_precision_and_upsampling(prec, eps, ups):
    # the candidate search (sizes c 2^k in increasing order, first admissible
    # split wins) against enumerating every candidate size below the answer
    import paper_2409_08090_gb300 as nl
    rng = np.random.default_rng(11)
    for nf in [1, 3, 50, 777] + [int(x) for x in np.exp(rng.uniform(np.log(1e3), np.log(8e6), 40))]:
        p = nl.ls_choose_params(nf, eps, prec, upsampling=ups)
        n, n1, n2 = p["n"], p["n1"], p["n2"]
        assert p["sigma"] == ups and n1 * n2 == n and _is_allowed(n)
        nmin = max(int(np.ceil(ups * nf - 1e-9)), 2 * p["width"], 64)
        assert n >= nmin
        # below 2^22 cells every c 2^k >= nmin with k >= 6 has an admissible split
        # (N1 = 32..512, N2 even and within the column limit), so none may be skipped
        if n <= 1 << 22:
            smaller = [c * 2 ** k for c in ODD for k in range(6, 40) if nmin <= c * 2 ** k < n]
            assert not smaller, (nf, n, smaller[:3])
        # the split is the most balanced admissible one among powers of two N1
        assert n1 & (n1 - 1) == 0 and n2 % 2 == 0
        bal = abs(np.log(n1) - np.log(n2))
        for k1 in range(5, 13):
            m1 = 1 << k1
            if n % m1 or m1 == n1 or (n // m1) % 2 or n // m1 > (25600 if prec == 1 else 12800):
                continue
            assert abs(np.log(m1) - np.log(n // m1)) >= bal - 1e-12, (nf, n1, m1)
