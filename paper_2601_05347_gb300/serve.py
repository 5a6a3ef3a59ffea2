"""Continuous-batching server over one device-resident index.

Requests (insert, delete, k-NN, range count, range list) arrive on any thread
and get an admission sequence number.  Semantics: a query sees exactly the
updates admitted before it.  A worker thread repeatedly takes every request
that has arrived and fits the device-memory budget, cuts the admitted sequence
into epochs at the updates, and for each epoch
  * coalesces its queries -- all k-NN requests with the same k into one
    psi_knn call, all range counts into one call, all range lists into one
    call -- and runs the groups concurrently on separate CUDA streams, with
    their host-to-device copies on those streams;
  * then applies the epoch's update on the main stream once the queries that
    read the previous tree state are done.
Requests that arrive while a round is on the GPU are admitted in the next
round, as slots and memory free up.  Results are copied back on the query
streams and each request's future is completed with its own slice.

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
    __slots__ = ("kind", "a", "b", "k", "arrival", "seq", "future", "done", "est_bytes")

    def __init__(self, kind: str, a: np.ndarray, b: np.ndarray | None = None, k: int = 0):
        assert kind in KINDS
        self.kind, self.a, self.b, self.k = kind, a, b, k
        self.arrival = 0.0
        self.done = 0.0
        self.seq = -1
        self.future = Future()
        n = len(a)
        self.est_bytes = {"insert": 160 * n, "delete": 120 * n, "knn": n * (8 + 12 * k + 64),
                          "count": 48 * n, "report": n * (48 + 4 * 2048)}[kind]


def _dev(a: np.ndarray, dev, stream) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    with torch.cuda.stream(stream):
        return torch.from_numpy(a).pin_memory().to(dev, non_blocking=True)


class Server:
    """Continuous-batching request loop around a psi.Index."""

    def __init__(self, index: "psi.Index", mem_budget: int | None = None, query_streams: int = 3):
        self.ix = index
        self.dev = torch.device("cuda", torch.cuda.current_device())
        free, _ = torch.cuda.mem_get_info(self.dev)
        self.budget = int(mem_budget if mem_budget is not None else 0.5 * free)
        self.main = torch.cuda.Stream(self.dev)
        self.qs = [torch.cuda.Stream(self.dev) for _ in range(query_streams)]
        self.pending = collections.deque()
        self.lock = threading.Condition()
        self.seq = 0
        self.stop_flag = False
        self.rounds = []  # (admitted, epochs) per round, for inspection
        self.worker = threading.Thread(target=self._loop, daemon=True)
        self.worker.start()

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

    # -- worker --------------------------------------------------------------
    def _admit(self):
        with self.lock:
            while not self.pending and not self.stop_flag:
                self.lock.wait()
            out, used = [], 0
            while self.pending and used + self.pending[0].est_bytes <= self.budget:
                r = self.pending.popleft()
                used += r.est_bytes
                out.append(r)
            return out

    def _loop(self):
        while True:
            batch = self._admit()
            if not batch:
                if self.stop_flag:
                    return
                continue
            epochs, cur = [], []
            for r in batch:
                if r.kind in ("insert", "delete"):
                    epochs.append((cur, r))
                    cur = []
                else:
                    cur.append(r)
            epochs.append((cur, None))
            self.rounds.append((len(batch), len(epochs)))
            try:
                for queries, update in epochs:
                    self._run_queries(queries)
                    if update is not None:
                        self._run_update(update)
            except Exception as e:  # fail every request of the round, keep serving
                for r in batch:
                    if not r.future.done():
                        r.future.set_exception(e)

    def _run_update(self, r: Request):
        s = self.main
        for q in self.qs:
            s.wait_stream(q)
        pts = _dev(r.a, self.dev, s)
        ids = _dev(r.b, self.dev, s)
        with torch.cuda.stream(s):
            if r.kind == "insert":
                self.ix.insert(pts, ids, stream=s)
                res = None
            else:
                nd = torch.zeros(1, dtype=torch.int64, device=self.dev)
                self.ix.delete(pts, ids, nd, stream=s)
                res = int(nd.item())
        r.done = time.perf_counter()
        r.future.set_result(res)

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
            x = _dev(cat, self.dev, s)
            with torch.cuda.stream(s):
                if kind == "knn":
                    ids, d2 = self.ix.knn(x, k, stream=s)
                    out = (ids.to("cpu", non_blocking=True), d2.to("cpu", non_blocking=True))
                elif kind == "count":
                    out = (self.ix.range_count(x, stream=s).to("cpu", non_blocking=True),)
                else:
                    off, rid = self.ix.range_report(x, stream=s)
                    out = (off.to("cpu", non_blocking=True), rid.to("cpu", non_blocking=True))
                ev = torch.cuda.Event()
                ev.record(s)
            launched.append((kind, rs, offs, out, ev))
        for kind, rs, offs, out, ev in launched:
            ev.synchronize()
            now = time.perf_counter()
            for j, r in enumerate(rs):
                a, b = offs[j], offs[j + 1]
                if kind == "knn":
                    res = (out[0][a:b].numpy().view(np.uint32), out[1][a:b].numpy())
                elif kind == "count":
                    res = out[0][a:b].numpy()
                else:
                    off = out[0].numpy()
                    res = (off[a:b + 1] - off[a], out[1][off[a]:off[b]].numpy().view(np.uint32))
                r.done = now
                r.future.set_result(res)


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


def percentiles(reqs, kind=None):
    lat = [(r.done - r.arrival) * 1e3 for r in reqs if kind is None or r.kind == kind]
    if not lat:
        return None
    return {"n": len(lat), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3)}
