"""ls_execute_noalloc: the periodogram entry point that allocates nothing.

It serves callers that cannot allocate device memory (programs whose device
memory belongs to another allocator or a fixed arena, loops that cannot
afford the synchronisation an allocation may bring): they cannot create an
ls_plan, so the library runs the same pipeline on a fixed scratch area it
reserves at load time.  The call is synchronous.  These tests call it through the C-ABI binding and compare its output
with the planned entry point, ls_execute, at the parity tolerances used
elsewhere (FP64 eps 1e-12: max |dP| <= 1e-9; FP32 eps 1e-6: relative l2
<= 1e-5), on consecutive calls that reuse the scratch area.  The file sorts
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2409_08090_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2409_08090_gb300 as m
    m.build.build()
    m.load_library()
    return m


def _device(s):
    import torch
    dev = torch.device("cuda:0")
    t = torch.tensor(s.t, dtype=torch.float64, device=dev)
    y = torch.tensor(s.y, dtype=torch.float64, device=dev)
    dy = None if s.dy is None else torch.tensor(s.dy, dtype=torch.float64, device=dev)
    return t, y, dy


def _noalloc(nl, s, eps, prec):
    import torch
    t, y, dy = _device(s)
    out = torch.full((s.nf,), float("nan"), dtype=torch.float64, device=t.device)
    st = nl.ls_execute_noalloc(t.data_ptr(), y.data_ptr(), dy.data_ptr() if dy is not None else None,
                               s.nd, s.f0, s.df, s.nf, eps, prec, out.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert st == nl.LS_OK, nl.ls_status_str(st)
    return out.cpu().numpy()


def _planned(nl, s, eps, prec):
    t, y, dy = _device(s)
    plan = nl.Plan(s.nd, s.nf, eps, prec)
    P = plan.execute(t, y, dy, s.f0, s.df).cpu().numpy()
    plan.close()
    return P


@pytest.mark.parametrize("prec,eps", [(1, 1e-6), (0, 1e-12)])
def test_noalloc_matches_ls_execute_on_consecutive_calls(nl, prec, eps):
    cases = [W.random_case(71, 3000, 9000),
             W.random_case(72, 1200, 5001, sort=False, unit_dy=True),
             W.single_small()]
    for s in cases + cases[:1]:          # the first case again after the others
        P = _noalloc(nl, s, eps, prec)
        R = _planned(nl, s, eps, prec)
        assert np.all(np.isfinite(P))
        if prec == 0:
            assert np.max(np.abs(P - R)) <= 1e-9
        else:
            assert np.linalg.norm(P - R) / np.linalg.norm(R) <= 1e-5
            assert np.max(np.abs(P - R)) <= 1e-4


def test_noalloc_rejects_requests_beyond_its_scratch(nl):
    import torch
    t = torch.linspace(0.0, 10.0, 64, dtype=torch.float64, device="cuda:0")
    y = torch.sin(t)
    out = torch.empty(64, dtype=torch.float64, device="cuda:0")
    big_nd = nl.ls_execute_noalloc(t.data_ptr(), y.data_ptr(), None, 16385, 0.1, 0.01, 64, 1e-9,
                                   0, out.data_ptr(), 0)
    big_nf = nl.ls_execute_noalloc(t.data_ptr(), y.data_ptr(), None, 64, 0.1, 0.01, 16385, 1e-9,
                                   0, out.data_ptr(), 0)
    assert big_nd == nl.LS_ERR_UNSUPPORTED and big_nf == nl.LS_ERR_UNSUPPORTED
    host = np.zeros(64)
    assert nl.ls_execute_noalloc(host.ctypes.data, y.data_ptr(), None, 64, 0.1, 0.01, 64, 1e-9, 0,
                                 out.data_ptr(), 0) == nl.LS_ERR_ARG
    # still usable afterwards
    assert nl.ls_execute_noalloc(t.data_ptr(), y.data_ptr(), None, 64, 0.1, 0.01, 64, 1e-9, 0,
                                 out.data_ptr(), 0) == nl.LS_OK
