"""Plans used from several host threads: a launch configuration chosen in one
thread (the shared-memory limit of the pass kernels) must not be undone by a
smaller plan executed from another thread."""
import threading

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


def _run(nl, s, prec, eps):
    import torch
    dev = torch.device("cuda:0")
    plan = nl.Plan(s.nd, s.nf, eps, prec)
    P = plan.execute(torch.tensor(s.t, device=dev), torch.tensor(s.y, device=dev),
                     torch.tensor(s.dy, device=dev), s.f0, s.df).cpu().numpy()
    plan.close()
    return P


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_large_then_small_in_another_thread_then_large(nl, prec, eps):
    big = W.random_case(501, 20000, 400_000, baseline=2000.0)
    small = W.random_case(502, 100, 500)
    first = _run(nl, big, prec, eps)
    box = {}

    def other():
        import torch
        torch.cuda.set_device(0)
        box["P"] = _run(nl, small, prec, eps)

    th = threading.Thread(target=other)
    th.start()
    th.join()
    again = _run(nl, big, prec, eps)
    assert box["P"].shape == (small.nf,) and np.all(np.isfinite(box["P"]))
    from tests.rerun_tolerance import assert_identical
    assert_identical(again, first)
