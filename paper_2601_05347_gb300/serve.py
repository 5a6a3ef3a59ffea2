"""Continuous-batching server over one device-resident index.

Requests (insert, delete, k-NN, range count, range list) arrive on any thread
and get an admission sequence number.  Semantics: a query sees exactly the
updates admitted before it.  A worker thread repeatedly takes every request
that has arrived and fits the device-memory budget, cuts the admitted sequence
into epochs at the updates, and for each epoch
  * coalesces its queries -- all k-NN requests with the same k into one
    psi_knn call, all range counts into one call, all range lists into one
    call -- and launches the groups on the query stream(s), inputs copied from
    pinned host memory on the same stream;
  * then applies the epoch's update on the main stream once the queries that
    read the previous tree state are done; consecutive inserts with no query
    between them are applied as one batch.
Requests that arrive while a round is on the GPU are admitted in the next
round, as slots and memory free up.  A finisher thread copies each group's
results into pinned host memory on a copy stream and completes every
request's future with its own slice (a numpy view of pinned memory, held until
the caller drops it), so the worker never waits for results.

The plain form (`serve_plain`) answers one request at a time in arrival order.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future

import numpy as np
import torch

from . import psi

KINDS = ("insert", "delete", "knn", "count", "report")


class Request:
    __slots__ = ("kind", "a", "b", "k", "arrival", "seq", "future", "done", "est_bytes", "t_admit", "t_launch",
                 "held")

    def __init__(self, kind: str, a: np.ndarray, b: np.ndarray | None = None, k: int = 0):
        assert kind in KINDS
        self.kind, self.a, self.b, self.k = kind, a, b, k
        self.arrival = 0.0
        self.done = 0.0
        self.t_admit = 0.0   # trace: taken by the worker
        self.t_launch = 0.0  # trace: its work enqueued on the device
        self.seq = -1
        self.held = False  # its est_bytes count against the server's budget
        self.future = Future()
        n = len(a)
        self.est_bytes = {"insert": 160 * n, "delete": 120 * n, "knn": n * (8 + 12 * k + 64),
                          "count": 48 * n, "report": n * (48 + 4 * 2048)}[kind]


def _dev(a: np.ndarray, dev, stream) -> torch.Tensor:
    """Host array -> device tensor, copied on `stream` (pageable source)."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    with torch.cuda.stream(stream):
        return torch.from_numpy(a).to(dev)


def _warm_pinned(total: int):
    """Puts pinned blocks of sizes 64 KiB, 128 KiB, ... (two of each, about
    `total` bytes in all) into the host caching allocator, so that staging and
    result copies later come from the cache rather than from fresh page-locked
    allocations, which are slow and stall the device."""
    keep, size = [], 1 << 16
    while 4 * size <= total:
        keep += [torch.empty(size, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        size <<= 1
    del keep


def plan_epochs(batch):
    """Splits an admitted round (arrival order) into epochs (queries, updates):
    the queries of an epoch run against the tree as every earlier update left
    it, then its updates apply -- one delete, or consecutive inserts with no
    query between them as one batch (the point set, and so every query result,
    is the same as inserting them one by one).  The last epoch has no update."""
    epochs, cur = [], []
    for r in batch:
        if r.kind in ("insert", "delete"):
            if (r.kind == "insert" and not cur and epochs and epochs[-1][1]
                    and epochs[-1][1][0].kind == "insert"):
                epochs[-1][1].append(r)
            else:
                epochs.append((cur, [r]))
            cur = []
        else:
            cur.append(r)
    epochs.append((cur, None))
    return epochs


class Server:
    """Continuous-batching request loop around a psi.Index."""

    def __init__(self, index: "psi.Index", mem_budget: int | None = None, query_streams: int = 1,
                 warm_pinned_bytes: int = 512 << 20):
        self.ix = index
        self.dev = torch.device("cuda", torch.cuda.current_device())
        free, _ = torch.cuda.mem_get_info(self.dev)
        self.budget = int(mem_budget if mem_budget is not None else 0.5 * free)
        self.main = torch.cuda.Stream(self.dev)
        self.qs = [torch.cuda.Stream(self.dev) for _ in range(query_streams)]
        self.copy = torch.cuda.Stream(self.dev)  # result copies: updates never wait on them
        _warm_pinned(warm_pinned_bytes)
        self.pending = collections.deque()
        self.lock = threading.Condition()
        self.inflight = 0  # est_bytes of admitted requests whose device memory is not yet released
        self.seq = 0
        self.stop_flag = False
        self.rounds = []  # (admitted, epochs) per round, for inspection
        self.completions = collections.deque()
        self.cv_done = threading.Condition()
        self.worker = threading.Thread(target=self._loop, daemon=True)
        self.finisher = threading.Thread(target=self._finish_loop, daemon=True)
        self.worker.start()
        self.finisher.start()

    # -- client side -------------------------------------------------------
    def submit(self, req: Request) -> Future:
        if req.est_bytes > self.budget:
            req.future.set_exception(MemoryError(f"request needs ~{req.est_bytes} B, budget is {self.budget} B"))
            return req.future
        with self.lock:
            req.arrival = time.perf_counter()
            req.seq = self.seq
            self.seq += 1
            self.pending.append(req)
            self.lock.notify()
        return req.future

    def close(self):
        with self.lock:
            self.stop_flag = True
            self.lock.notify()
        self.worker.join()
        with self.cv_done:
            self.completions.append(None)
            self.cv_done.notify()
        self.finisher.join()

    # -- worker --------------------------------------------------------------
    def _admit(self):
        """Takes the pending requests, in arrival order, that fit the budget
        next to the device memory still held by earlier rounds (query results
        not yet copied back); waits while none fits."""
        with self.lock:
            while True:
                while not self.pending and not self.stop_flag:
                    self.lock.wait()
                out, used = [], 0
                now = time.perf_counter()
                while self.pending and self.inflight + used + self.pending[0].est_bytes <= self.budget:
                    r = self.pending.popleft()
                    used += r.est_bytes
                    r.t_admit = now
                    r.held = True
                    out.append(r)
                if out or not self.pending or self.stop_flag and not self.inflight:
                    self.inflight += used
                    return out
                self.lock.wait()  # the finisher releases memory and notifies

    def _release(self, rs):
        """Returns the budget share of requests whose device memory is freed."""
        freed = 0
        for r in rs:
            if r.held:
                r.held = False
                freed += r.est_bytes
        if freed:
            with self.lock:
                self.inflight -= freed
                self.lock.notify_all()

    def _loop(self):
        while True:
            batch = self._admit()
            if not batch:
                if self.stop_flag:
                    return
                continue
            epochs = plan_epochs(batch)
            self.rounds.append((len(batch), len(epochs)))
            try:
                for queries, updates in epochs:
                    self._run_queries(queries)
                    if updates:
                        self._run_update(updates)
                        self._release(updates)  # done synchronously: its inputs are freed
            except Exception as e:  # fail every request of the round, keep serving
                for r in batch:
                    if not r.future.done():
                        r.future.set_exception(e)
                self._release([r for r in batch if r.future.done() and r.future.exception() is not None])

    def _to_dev(self, a: np.ndarray, s) -> torch.Tensor:
        """Host array -> device: a pinned copy (host caching allocator), sent
        asynchronously on stream s; the pinned block is not reused before that
        copy is done."""
        a = np.ascontiguousarray(a)
        if a.dtype == np.uint32:
            a = a.view(np.int32)
        h = torch.from_numpy(a).pin_memory()
        with torch.cuda.stream(s):
            return h.to(self.dev, non_blocking=True)

    def _run_update(self, rs):
        s = self.main
        for q in self.qs:
            s.wait_stream(q)
        r = rs[0]
        if len(rs) > 1:  # consecutive inserts: one batch
            a = np.concatenate([x.a for x in rs])
            b = np.concatenate([x.b for x in rs])
        else:
            a, b = r.a, r.b
        pts = self._to_dev(a, s)
        ids = self._to_dev(b, s)
        now = time.perf_counter()
        for x in rs:
            x.t_launch = now
        with torch.cuda.stream(s):
            if r.kind == "insert":
                self.ix.insert(pts, ids, stream=s)
                res = None
            else:
                nd = torch.zeros(1, dtype=torch.int64, device=self.dev)
                self.ix.delete(pts, ids, nd, stream=s)
                res = int(nd.item())
        now = time.perf_counter()
        for x in rs:
            x.done = now
            x.future.set_result(res)

    def _run_queries(self, reqs):
        if not reqs:
            return
        groups = collections.OrderedDict()
        for r in reqs:
            groups.setdefault((r.kind, r.k), []).append(r)
        launched = []
        for gi, ((kind, k), rs) in enumerate(groups.items()):
            s = self.qs[gi % len(self.qs)]
            s.wait_stream(self.main)  # the tree state of this epoch
            cat = np.concatenate([r.a for r in rs])
            offs = np.cumsum([0] + [len(r.a) for r in rs])
            x = self._to_dev(cat, s)
            with torch.cuda.stream(s):
                if kind == "knn":
                    out = self.ix.knn(x, k, stream=s)
                elif kind == "count":
                    out = (self.ix.range_count(x, stream=s),)
                else:
                    out = self.ix.range_report(x, stream=s)
                ev = torch.cuda.Event()
                ev.record(s)
            now = time.perf_counter()
            for r in rs:
                r.t_launch = now
            launched.append((kind, rs, offs, out, ev, x))
        # results are copied back and handed out by the finisher thread, so
        # the worker can launch the next epoch meanwhile
        with self.cv_done:
            self.completions.append(launched)
            self.cv_done.notify()

    def _finish_loop(self):
        while True:
            with self.cv_done:
                while not self.completions:
                    self.cv_done.wait()
                launched = self.completions.popleft()
            if launched is None:
                return
            self._finish(launched)

    def _finish(self, launched):
        for kind, rs, offs, dout, ev, _keep in launched:
            # device-to-host copies after the group's kernels, into pinned
            # blocks of the host caching allocator; every request's result is
            # a view of its slice (the block is reused once all views are gone)
            self.copy.wait_event(ev)
            with torch.cuda.stream(self.copy):
                out = []
                for t in dout:
                    h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                    h.copy_(t, non_blocking=True)
                    out.append(h.numpy())
            self.copy.synchronize()
            now = time.perf_counter()
            for j, r in enumerate(rs):
                a, b = offs[j], offs[j + 1]
                if kind == "knn":
                    res = (out[0][a:b].view(np.uint32), out[1][a:b])
                elif kind == "count":
                    res = out[0][a:b]
                else:
                    off = out[0]
                    res = (off[a:b + 1] - off[a], out[1][off[a]:off[b]].view(np.uint32))
                r.done = now
                r.future.set_result(res)
            self._release(rs)  # the group's results are on the host


def serve_plain(index: "psi.Index", req: Request):
    """The plain form: one request, synchronously, on the current stream."""
    dev = torch.device("cuda", torch.cuda.current_device())
    s = torch.cuda.current_stream()
    x = _dev(req.a, dev, s)
    if req.kind in ("insert", "delete"):
        ids = _dev(req.b, dev, s)
        if req.kind == "insert":
            index.insert(x, ids)
            return None
        nd = torch.zeros(1, dtype=torch.int64, device=dev)
        index.delete(x, ids, nd)
        return int(nd.item())
    if req.kind == "knn":
        i, d = index.knn(x, req.k)
        return i.cpu().numpy().view(np.uint32), d.cpu().numpy()
    if req.kind == "count":
        return index.range_count(x).cpu().numpy()
    off, rid = index.range_report(x)
    return off.cpu().numpy(), rid.cpu().numpy().view(np.uint32)


def trace_breakdown(reqs, kind=None):
    """Median milliseconds from arrival to admission, admission to launch, and
    launch to completion (served requests only)."""
    rs = [r for r in reqs if (kind is None or r.kind == kind) and r.t_admit > 0]
    if not rs:
        return None
    med = lambda v: round(float(np.median(v)) * 1e3, 3)
    return {"n": len(rs), "queue_ms": med([r.t_admit - r.arrival for r in rs]),
            "admit_to_launch_ms": med([r.t_launch - r.t_admit for r in rs]),
            "launch_to_done_ms": med([r.done - r.t_launch for r in rs])}


def percentiles(reqs, kind=None):
    lat = [(r.done - r.arrival) * 1e3 for r in reqs if kind is None or r.kind == kind]
    if not lat:
        return None
    return {"n": len(lat), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3)}
