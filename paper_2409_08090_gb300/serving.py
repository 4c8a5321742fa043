"""Serving: periodogram requests admitted as they arrive, batched continuously.

A request is one series (t, y, dy) with its frequency grid and a precision.
`Scheduler` is the host-side policy, free of CUDA so it can be tested alone:
FIFO admission under a device-memory budget, grouping of admitted requests by
(precision, tolerance) into batches, cancellation before admission, and the
bookkeeping of bytes in flight.  `PeriodogramServer` drives the GPU: one loop
thread keeps a plan per (precision, tolerance) and per stream resident (their
fine-grid tables and workspaces stay allocated between batches), launches each
batch through `ls_execute_batch` on one of several CUDA streams, and admits the
next requests while earlier batches are still running, so their work overlaps
on the device.  Latency (arrival to result) and throughput are recorded per
request.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import itertools
import threading
import time
from dataclasses import dataclass, field

import numpy as np

__all__ = ["Request", "Scheduler", "PeriodogramServer", "request_bytes", "lane_bytes"]

_ids = itertools.count()


def request_bytes(nd: int, nf: int, precision: str) -> int:
    """Device bytes a request holds while in flight outside the plans: its
    inputs (t, y, dy) and its output.  Its fine grids and point records live in
    the serving plans' reserved batch workspaces, which the server counts
    separately (``Scheduler.reserved``)."""
    return int(24 * nd + 8 * nf)


def lane_bytes(nd: int, nf: int, precision: str, eps: float) -> int:
    """Upper bound of the batch-workspace bytes one series occupies alone in a
    launch (its three fine grids, four point-record sets, bin and chunk
    tables), from the grid the library chooses for it."""
    import paper_2409_08090_gb300 as nl
    q = nl.ls_choose_params(int(nf), float(eps), nl.LS_FP32 if precision == "fp32" else nl.LS_FP64,
                            int(nd))
    cx = 8 if precision == "fp32" else 16
    recb = 28 if precision == "fp32" else 48
    n, nbins = int(q["n"]), int(q["n1"])
    return int(3 * n * cx + 4 * (recb * nd + 1280) + 4 * (4 * nbins + 2)
               + 4 * (nd // 2048 + 1) * 2 * nbins + 12 * nbins + 8 * 256)


@dataclass
class Request:
    t: np.ndarray
    y: np.ndarray
    dy: np.ndarray | None
    f0: float
    df: float
    nf: int
    precision: str = "fp32"
    eps: float = 1e-6
    mode: int = 0           # normalisation and model flags (the C-ABI's norm word)
    id: int = field(default_factory=lambda: next(_ids))
    arrival: float = field(default_factory=time.perf_counter)
    future: cf.Future = field(default_factory=cf.Future)
    done: float | None = None

    @property
    def nd(self) -> int:
        return int(self.t.shape[0])

    @property
    def nbytes(self) -> int:
        return request_bytes(self.nd, self.nf, self.precision)

    @property
    def key(self):
        return (self.precision, float(self.eps), int(self.mode))


class Scheduler:
    """Admission and batching policy (host only).

    * FIFO: a request is admitted only after every earlier one; when the head
      does not fit the free budget (budget - reserved - in use), admission
      waits for memory to be released (no overtaking, so large requests are
      not starved).
    * A request larger than the whole budget is rejected with MemoryError.
    * Admitted requests with the same (precision, eps, model) form a batch of at most
      `max_batch` series; `next_batch` returns the largest group first.
    * Cancelled requests (future.cancel() before admission) are dropped.
    """

    def __init__(self, budget_bytes: int, max_batch: int = 4096):
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.in_use = 0
        self.reserved = 0       # bytes held outside requests (the server's plans)
        self.pending: collections.deque[Request] = collections.deque()
        self.admitted: list[Request] = []
        self.lock = threading.Lock()

    def submit(self, req: Request) -> cf.Future:
        if req.nbytes > self.budget:
            req.future.set_exception(MemoryError(
                f"request needs {req.nbytes} B of device memory, budget {self.budget} B"))
            return req.future
        with self.lock:
            self.pending.append(req)
        return req.future

    def _admit(self):
        while self.pending:
            head = self.pending[0]
            if head.future.cancelled():
                self.pending.popleft()
                continue
            if self.reserved + self.in_use + head.nbytes > self.budget:
                break
            if not head.future.set_running_or_notify_cancel():
                self.pending.popleft()
                continue
            self.pending.popleft()
            self.in_use += head.nbytes
            self.admitted.append(head)

    def next_batch(self) -> list[Request]:
        """Admit what fits, then take one batch of admitted requests."""
        with self.lock:
            self._admit()
            if not self.admitted:
                return []
            groups = collections.OrderedDict()
            for r in self.admitted:
                groups.setdefault(r.key, []).append(r)
            key = max(groups, key=lambda k: len(groups[k]))
            batch = groups[key][: self.max_batch]
            taken = set(id(r) for r in batch)
            self.admitted = [r for r in self.admitted if id(r) not in taken]
            return batch

    def release(self, batch: list[Request]):
        with self.lock:
            for r in batch:
                self.in_use -= r.nbytes

    def set_reserved(self, nbytes: int):
        """Bytes held outside the requests (resident plans); admission counts
        them against the budget."""
        with self.lock:
            self.reserved = int(nbytes)

    def idle(self) -> bool:
        with self.lock:
            return not self.pending and not self.admitted


class _Slot:
    """One CUDA stream with its own plans (a plan is not thread-safe and owns
    one workspace, so each stream has its own)."""

    def __init__(self, device: int):
        import torch
        self.stream = torch.cuda.Stream(device=device)
        self.plans = {}
        self.batch = None
        self.done_event = None
        self.out_host = None
        self.plan = None
        self.keep = None        # device tensors alive until the batch completes
        self.pin_in = None      # pinned input staging reused across batches
        self.pin_out = None     # pinned output staging of small batches
        self.views = False      # results of the batch in flight are views of its buffer

    def pinned(self, which: str, n: int):
        import torch
        buf = getattr(self, which)
        if buf is None or buf.numel() < n:
            buf = torch.empty(max(n, 1 << 16) * 5 // 4, dtype=torch.float64).pin_memory()
            setattr(self, which, buf)
        return buf[:n]


class PeriodogramServer:
    """Continuous-batching periodogram server on one GPU.

    submit() returns a Future resolved with the float64 power: a numpy array
    (results="host": a view of the batch's pinned host buffer, which lives as
    long as any of its views), or a view of the batch's CUDA tensor
    (results="device", no host copy at all).
    `streams` batches can be on the GPU at once; requests arriving meanwhile
    are admitted (memory permitting) into the next batch.
    """

    def __init__(self, device: int = 0, memory_budget: int = 60 << 30, streams: int = 2,
                 max_batch: int = 4096, results: str = "host",
                 plan_workspace_bytes: int | None = None):
        import torch

        import paper_2409_08090_gb300 as nl
        self._nl = nl
        nl.load_library()
        self.device = int(device)
        torch.cuda.set_device(self.device)
        if results not in ("host", "device"):
            raise ValueError("results must be 'host' (numpy arrays) or 'device' (CUDA tensors)")
        self.results = results
        # Host results are views of a fresh pinned buffer per batch (torch keeps
        # freed pinned blocks cached, so after warm-up this costs no allocation;
        # a buffer stays pinned while any of its views lives).  Batches of at most
        # copy_limit output bytes are copied out per request into plain arrays
        # instead; copying was measured to saturate the server loop at 5000 req/s
        # (3.5k/s, p50 0.8 s, against 4.9k/s, p50 34 ms with views), so 0.
        self.copy_limit = 0
        self.sched = Scheduler(memory_budget, max_batch)
        self.budget = int(memory_budget)
        # Each resident plan (one per stream and (precision, eps)) reserves a
        # fixed batch workspace when it is created, so serving never grows or
        # reallocates one; its bytes, with its grid classes' tables, are counted
        # against the budget before any request.  A lane holds a quarter.
        self.plan_ws = int(plan_workspace_bytes if plan_workspace_bytes is not None
                           else min(1 << 30, max(64 << 20, self.budget // 16)))
        self.peak_device_bytes = 0    # torch allocations + plans, sampled per batch
        self.slots = [_Slot(self.device) for _ in range(max(1, int(streams)))]
        self.cv = threading.Condition()
        self.stop = False
        # (arrival, done) of finished requests, for stats(); the requests
        # themselves are not kept, so a result lives only as long as its caller
        # holds it (host results pin their batch's buffer until then)
        self.completed: list[tuple[float, float]] = []
        self.batches = 0
        self.thread = threading.Thread(target=self._loop, name="periodogram-server", daemon=True)
        self.thread.start()

    # ---- client side -------------------------------------------------------
    def submit(self, t, y, dy, f0: float, df: float, nf: int, precision: str = "fp32",
               eps: float | None = None, normalization: str = "standard",
               fit_mean: bool = True, center_data: bool = True) -> cf.Future:
        try:
            mode = self._nl.mode_word(normalization, fit_mean, center_data)
        except ValueError as exc:
            fut = cf.Future()
            fut.set_exception(exc)
            return fut
        t = np.ascontiguousarray(t, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        dy = None if dy is None else np.ascontiguousarray(np.broadcast_to(dy, t.shape),
                                                          dtype=np.float64)
        eps = (1e-6 if precision == "fp32" else 1e-9) if eps is None else float(eps)
        req = Request(t, y, dy, float(f0), float(df), int(nf), precision, eps, mode)
        bad = (t.ndim != 1 or t.shape != y.shape or t.shape[0] < 2 or req.nf < 1
               or not (req.df > 0) or not np.all(np.isfinite(t)) or not np.all(np.isfinite(y))
               or (dy is not None and not np.all(dy > 0)))
        if bad:
            req.future.set_exception(ValueError("invalid request"))
            return req.future
        try:
            need = lane_bytes(req.nd, req.nf, precision, eps)
        except Exception as exc:          # no admissible grid for this request
            req.future.set_exception(exc)
            return req.future
        if need > self.plan_ws // 4:
            req.future.set_exception(MemoryError(
                f"request needs {need} B of batch workspace, a plan lane holds {self.plan_ws // 4} B"))
            return req.future
        self.sched.submit(req)
        with self.cv:
            self.cv.notify()
        return req.future

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify()
        self.thread.join()
        for s in self.slots:
            for p in s.plans.values():
                p.close()

    def drain(self, timeout: float | None = None):
        t0 = time.perf_counter()
        while not self.sched.idle() or any(s.batch for s in self.slots):
            if timeout is not None and time.perf_counter() - t0 > timeout:
                raise TimeoutError("server did not drain")
            time.sleep(0.001)

    def plan_bytes(self) -> int:
        """Device bytes the resident plans hold (workspaces and tables)."""
        return sum(p.device_bytes() for sl in self.slots for p in sl.plans.values())

    def stats(self) -> dict:
        lat = np.array([done - arrival for arrival, done in self.completed])
        if lat.size == 0:
            return {"requests": 0}
        span = max(d for _, d in self.completed) - min(a for a, _ in self.completed)
        return {"requests": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "periodograms_per_s": float(lat.size / span) if span > 0 else None,
                "batches": self.batches, "plan_bytes": self.sched.reserved,
                "peak_device_bytes": self.peak_device_bytes, "budget": self.budget}

    def _account(self):
        """Refresh the plans' bytes in the scheduler and the high-water mark of
        the device bytes this server holds (torch allocations + plans)."""
        import torch
        reserved = self.plan_bytes()
        self.sched.set_reserved(reserved)
        used = int(torch.cuda.memory_allocated(self.device)) + reserved
        self.peak_device_bytes = max(self.peak_device_bytes, used)

    # ---- GPU loop ----------------------------------------------------------
    def _plan(self, slot: _Slot, key):
        pk = key[:2]            # (precision, eps): the model word is per call
        p = slot.plans.get(pk)
        if p is None:
            # plans of other keys on this stream are closed first when the new
            # one's reservation would not fit the budget beside what is in use
            while (slot.plans and self.sched.reserved + self.sched.in_use + self.plan_ws
                   > self.budget):
                _, old = slot.plans.popitem()
                old.close()
                self.sched.set_reserved(self.plan_bytes())
            p = self._nl.Plan(2, 1, key[1], key[0], device=self.device,
                              batch_workspace_bytes=self.plan_ws)
            p.reserve_batch()
            slot.plans[pk] = p
            self._account()
        return p

    def _launch(self, slot: _Slot, batch: list[Request]):
        import torch
        nl = self._nl
        offsets = np.zeros(len(batch) + 1, dtype=np.int64)
        offsets[1:] = np.cumsum([r.nd for r in batch])
        nfs = np.array([r.nf for r in batch], dtype=np.int64)
        n = int(offsets[-1])
        host = slot.pinned("pin_in", 3 * n)
        hv = host.numpy()
        for r, a in zip(batch, offsets[:-1]):
            hv[a:a + r.nd] = r.t
            hv[n + a:n + a + r.nd] = r.y
            hv[2 * n + a:2 * n + a + r.nd] = 1.0 if r.dy is None else r.dy
        plan = self._plan(slot, batch[0].key)
        with torch.cuda.stream(slot.stream):
            dev = host.to(self.device, non_blocking=True)
            out = torch.empty(int(nfs.sum()), dtype=torch.float64, device=self.device)
            word = batch[0].mode
            _, out_off = plan.execute_batch(
                dev[:n], dev[n:2 * n], dev[2 * n:], offsets, [r.f0 for r in batch],
                [r.df for r in batch], nfs, out=out, sync=False,
                normalization=nl.NORMALIZATIONS[word & 0xFF],
                fit_mean=not (word & nl.LS_NO_FIT_MEAN),
                center_data=not (word & nl.LS_NO_CENTER))
            if self.results == "host":
                if out.numel() * 8 <= self.copy_limit:
                    # small batch: the slot's reused pinned buffer, copied out per request
                    out_host = slot.pinned("pin_out", out.numel())
                    slot.views = False
                else:
                    # large batch: a fresh pinned buffer (torch caches pinned
                    # blocks) handed out as views, so no per-request host copy;
                    # it returns to the cache when its last view is dropped
                    out_host = torch.empty(out.numel(), dtype=torch.float64, pin_memory=True)
                    slot.views = True
                out_host.copy_(out, non_blocking=True)
            else:
                out_host = out
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        slot.batch = batch
        slot.done_event = ev
        slot.out_host = (out_host, out_off)
        slot.plan = plan
        slot.keep = (host, dev, out)
        self.batches += 1
        self._account()

    def _finish(self, slot: _Slot):
        nl = self._nl
        batch, (out_host, out_off) = slot.batch, slot.out_host
        st = nl.ls_sync(slot.plan.handle)
        now = time.perf_counter()
        res = out_host.numpy() if self.results == "host" else out_host
        for r, o in zip(batch, out_off):
            r.done = now
            if st != nl.LS_OK:
                r.future.set_exception(nl.LSError(st, "batch"))
            elif self.results == "host":
                r.future.set_result(res[o:o + r.nf] if slot.views else res[o:o + r.nf].copy())
            else:
                r.future.set_result(res[int(o):int(o) + r.nf])
        self.completed.extend((r.arrival, r.done) for r in batch)
        slot.batch = slot.done_event = slot.out_host = slot.keep = None
        self._account()        # a new grid class may have added tables
        self.sched.release(batch)

    def _loop(self):
        import torch
        torch.cuda.set_device(self.device)
        while True:
            progressed = False
            for slot in self.slots:
                if slot.batch is not None and slot.done_event.query():
                    self._finish(slot)
                    progressed = True
            for slot in self.slots:
                if slot.batch is None:
                    batch = self.sched.next_batch()
                    if batch:
                        try:
                            self._launch(slot, batch)
                        except Exception as exc:      # pragma: no cover - reported per request
                            for r in batch:
                                r.future.set_exception(exc)
                            self.sched.release(batch)
                            slot.batch = None
                        progressed = True
            busy = any(s.batch is not None for s in self.slots)
            with self.cv:
                if self.stop and not busy and self.sched.idle():
                    return
                if not progressed:
                    self.cv.wait(timeout=0.0005 if busy else 0.01)
