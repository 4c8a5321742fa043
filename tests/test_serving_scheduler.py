"""Host-side serving policy (no GPU): FIFO admission under a device-memory
budget, budget exhaustion, cancellation before admission, grouping by
(precision, tolerance), and concurrent submitters."""
import threading

import numpy as np
import pytest

from paper_2409_08090_gb300.serving import Request, Scheduler, request_bytes


def _req(nd=100, nf=1200, precision="fp32", eps=1e-6):
    t = np.linspace(0, 10, nd)
    return Request(t, np.sin(t), None, 0.1, 0.01, nf, precision, eps)


def test_fifo_admission_waits_for_memory():
    a, b, c = _req(nf=1000), _req(nf=5000), _req(nf=1000)
    budget = a.nbytes + b.nbytes - 1          # a and b do not fit together
    s = Scheduler(budget)
    for r in (a, b, c):
        s.submit(r)
    first = s.next_batch()
    assert first == [a]                       # b waits; c may not overtake it
    assert s.next_batch() == []
    s.release(first)
    second = s.next_batch()
    assert second == [b]
    s.release(second)
    assert s.next_batch() == [c]
    assert s.in_use == c.nbytes


def test_oversized_request_is_rejected():
    s = Scheduler(1000)
    r = _req(nd=1000, nf=100_000)
    fut = s.submit(r)
    with pytest.raises(MemoryError):
        fut.result(timeout=1)
    assert s.idle()


def test_cancelled_requests_are_dropped():
    s = Scheduler(1 << 30)
    rs = [_req() for _ in range(5)]
    for r in rs:
        s.submit(r)
    assert rs[1].future.cancel() and rs[3].future.cancel()
    batch = s.next_batch()
    assert batch == [rs[0], rs[2], rs[4]]
    assert all(r.future.running() for r in batch)
    # admitted requests can no longer be cancelled
    assert not batch[0].future.cancel()


def test_batches_group_by_precision_and_tolerance():
    s = Scheduler(1 << 30, max_batch=3)
    rs = [_req(precision="fp32", eps=1e-6) for _ in range(5)] + \
         [_req(precision="fp64", eps=1e-9) for _ in range(2)]
    for r in rs:
        s.submit(r)
    b1 = s.next_batch()
    assert len(b1) == 3 and all(r.key == ("fp32", 1e-6, 0) for r in b1)
    b2 = s.next_batch()
    assert len(b2) == 2 and all(r.key == b2[0].key for r in b2)
    b3 = s.next_batch()
    assert len(b3) == 2 and {r.key for r in b2 + b3} == {("fp32", 1e-6, 0), ("fp64", 1e-9, 0)}
    assert s.next_batch() == []


def test_concurrent_submitters_and_release_balance():
    s = Scheduler(50 * request_bytes(100, 1200, "fp32"), max_batch=7)
    subs = []

    def worker(k):
        for i in range(40):
            r = _req()
            subs.append(r)
            s.submit(r)

    th = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for x in th:
        x.start()
    seen = []
    while len(seen) < 160:
        b = s.next_batch()
        assert s.in_use <= s.budget
        seen.extend(b)
        s.release(b)
    for x in th:
        x.join()
    assert len(set(id(r) for r in seen)) == 160
    assert s.in_use == 0 and s.idle()


def test_request_bytes_count_inputs_and_output():
    # t, y, dy in and the power out (FP64); grids live in the plans' workspaces
    assert request_bytes(1000, 12000, "fp32") == 24 * 1000 + 8 * 12000
    assert request_bytes(1000, 12000, "fp64") == request_bytes(1000, 12000, "fp32")


def test_reserved_bytes_count_against_the_budget():
    a = _req()
    s = Scheduler(a.nbytes * 3)
    s.set_reserved(a.nbytes * 2 + 1)            # resident plans leave room for less than one
    s.submit(a)
    assert s.next_batch() == []
    s.set_reserved(a.nbytes * 2)
    assert s.next_batch() == [a]


def test_model_variants_are_batched_apart():
    s = Scheduler(1 << 30)
    a, b = _req(), _req()
    b.mode = 0x103                      # psd, no fitted mean
    s.submit(a)
    s.submit(b)
    first, second = s.next_batch(), s.next_batch()
    assert len(first) == 1 and len(second) == 1 and first[0].key != second[0].key


def test_server_stats_from_timestamps_only():
    # the server keeps (arrival, done) pairs, not the requests (whose futures
    # hold the results): stats come from the timestamps alone
    import types

    from paper_2409_08090_gb300.serving import PeriodogramServer
    fake = types.SimpleNamespace(completed=[(0.0, 0.001), (0.5, 0.502), (1.0, 1.010)],
                                 batches=2, sched=types.SimpleNamespace(reserved=7),
                                 peak_device_bytes=11, budget=13)
    st = PeriodogramServer.stats(fake)
    assert st["requests"] == 3 and st["batches"] == 2
    assert (st["plan_bytes"], st["peak_device_bytes"], st["budget"]) == (7, 11, 13)
    assert st["p50_ms"] == pytest.approx(2.0)
    assert st["periodograms_per_s"] == pytest.approx(3 / 1.010)
    assert np.percentile([1.0, 2.0, 10.0], 99) == pytest.approx(st["p99_ms"])
    assert PeriodogramServer.stats(types.SimpleNamespace(completed=[], batches=0)) == \
        {"requests": 0}
