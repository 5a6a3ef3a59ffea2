"""Thin Python binding of the C ABI in include/psi.h.

Argument marshalling only: every step of build, update and query runs in the
CUDA library (_build/libpsi.so).  PyTorch provides device memory (tensors) and
streams.  There is no CPU fallback: if the library is missing, every call
raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _build

SPAC_Z, SPAC_H, PORTH = 0, 1, 2
KINDS = {"spac_z": SPAC_Z, "spac_h": SPAC_H, "porth": PORTH}
REPORT_SORTED = 1

OK, ERR_INVALID, ERR_RANGE, ERR_OOM, ERR_CAPACITY, ERR_DEVICE_TIMEOUT, ERR_CUDA = range(7)
_STATUS = {1: "PSI_ERR_INVALID", 2: "PSI_ERR_RANGE", 3: "PSI_ERR_OOM", 4: "PSI_ERR_CAPACITY",
           5: "PSI_ERR_DEVICE_TIMEOUT", 6: "PSI_ERR_CUDA"}


class PsiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("kind", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("coord_bits", ctypes.c_int32), ("fanout", ctypes.c_int32), ("radix_bits", ctypes.c_int32)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library not built: {_build.LIB} (run __graft_entry__.build())")
        L = ctypes.CDLL(_build.LIB)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        st = ctypes.c_int
        sig = {
            "psi_build": (st, [P, P, P, i64, P, P]),
            "psi_insert_batch": (st, [P, P, P, i64, P]),
            "psi_delete_batch": (st, [P, P, P, i64, P, P]),
            "psi_knn": (st, [P, P, i64, i32, P, P, P]),
            "psi_range_count": (st, [P, P, i64, P, P]),
            "psi_range_report": (st, [P, P, i64, P, P, i64, P, i32, P]),
            "psi_sync": (st, [P, P]),
            "psi_destroy": (st, [P]),
            "psi_size": (i64, [P]),
            "psi_num_leaves": (i64, [P]),
            "psi_num_nodes": (i64, [P]),
            "psi_last_error": (ctypes.c_char_p, []),
            "psi_export_leaves": (st, [P, P, P, P, P, P, P]),
            "psi_export_points": (st, [P, P, P, P, P, P]),
            "psi_export_nodes": (st, [P, P, P, P, P, P, P, P]),
            "psi_encode": (st, [P, P, i64, P, P]),
            "psi_sort_pairs": (st, [P, P, i64, i32, P]),
            "psi_knn_instrumented": (st, [P, P, i64, i32, P, P, P, P]),
            "psi_sort_pairs_noalloc": (st, [P, P, i64, i32, P]),
            "psi_test_sort_withheld_tile": (st, [P, P, i64, i64, ctypes.c_uint32, P]),
            "psi_batch_create": (st, [P, P, i32, i32, P, P]),
            "psi_batch_build": (st, [P, P, P, P]),
            "psi_batch_knn_reserve": (st, [P, i64, P]),
            "psi_batch_knn": (st, [P, P, P, i64, i32, P, P, P]),
            "psi_batch_knn_instrumented": (st, [P, P, P, i64, i32, P, P, P, P]),
            "psi_batch_sync": (st, [P, P]),
            "psi_batch_destroy": (st, [P]),
            "psi_batch_num_leaves": (i64, [P, i32]),
            "psi_batch_export_index": (st, [P, i32, P, P, P, P, P]),
            "psi_forth_build": (st, [P, P, P, i64, P, P]),
            "psi_forth_insert": (st, [P, P, P, i64, P]),
            "psi_forth_delete": (st, [P, P, P, i64, P, P]),
            "psi_forth_knn": (st, [P, P, i64, i32, P, P, P]),
            "psi_forth_range_count": (st, [P, P, i64, P, P]),
            "psi_forth_size": (i64, [P]),
            "psi_forth_num_nodes": (i64, [P]),
            "psi_forth_export": (st, [P, P, P, P, P, P, P, P, P, P]),
            "psi_forth_sync": (st, [P, P]),
            "psi_forth_destroy": (None, [P]),
            "psi_launch_count": (i64, []),
            "psi_profile_enable": (None, [ctypes.c_int]),
            "psi_profile_reset": (None, []),
            "psi_profile_read": (ctypes.c_int, [ctypes.c_char_p, P, P]),
            "psi_profile_dump": (ctypes.c_int, [ctypes.c_char_p, i64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != OK:
        raise PsiError(status, lib().psi_last_error().decode())


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _u32(t: torch.Tensor) -> torch.Tensor:
    """4-byte integer tensor viewed for the ABI (uint32 bit pattern)."""
    if t.element_size() != 4:
        raise ValueError("ids must be a 4-byte integer tensor")
    return t


class Index:
    """A device-resident spatial index (SPaC-Z, SPaC-H or P-Orth)."""

    def __init__(self, pts: torch.Tensor, ids: torch.Tensor, *, kind: int | str = SPAC_Z, leaf_size: int = 32,
                 coord_bits: int | None = None, fanout: int = 32, radix_bits: int = 0, stream=None):
        if isinstance(kind, str):
            kind = KINDS[kind]
        dim = int(pts.shape[1]) if pts.dim() == 2 else 2
        if coord_bits is None:
            coord_bits = 30 if dim == 2 else 21
        self.dim, self.kind, self.leaf_size, self.coord_bits, self.fanout = dim, kind, leaf_size, coord_bits, fanout
        self.cfg = Config(dim, kind, leaf_size, coord_bits, fanout, radix_bits)
        self._ids_per_box = 64.0  # running estimate that sizes range_report outputs
        h = ctypes.c_void_p()
        pts = pts.contiguous()
        ids = _u32(ids).contiguous()
        _check(lib().psi_build(ctypes.byref(self.cfg), _ptr(pts), _ptr(ids), int(pts.shape[0]), _stream(stream),
                               ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().psi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self) -> int:
        return int(lib().psi_size(self._h))

    @property
    def num_leaves(self) -> int:
        return int(lib().psi_num_leaves(self._h))

    @property
    def num_nodes(self) -> int:
        return int(lib().psi_num_nodes(self._h))

    def sync(self, stream=None):
        _check(lib().psi_sync(self._h, _stream(stream)))

    def insert(self, pts: torch.Tensor, ids: torch.Tensor, stream=None):
        pts, ids = pts.contiguous(), _u32(ids).contiguous()
        _check(lib().psi_insert_batch(self._h, _ptr(pts), _ptr(ids), int(pts.shape[0]), _stream(stream)))

    def delete(self, pts: torch.Tensor, ids: torch.Tensor, num_deleted: torch.Tensor | None = None, stream=None):
        pts, ids = pts.contiguous(), _u32(ids).contiguous()
        _check(lib().psi_delete_batch(self._h, _ptr(pts), _ptr(ids), int(pts.shape[0]), _ptr(num_deleted),
                                      _stream(stream)))

    def knn(self, q: torch.Tensor, k: int, out_ids: torch.Tensor | None = None, out_d2: torch.Tensor | None = None,
            stream=None):
        q = q.contiguous()
        nq = int(q.shape[0])
        if out_ids is None:
            out_ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        if out_d2 is None:
            out_d2 = torch.empty((nq, k), dtype=torch.int64, device=q.device)
        _check(lib().psi_knn(self._h, _ptr(q), nq, k, _ptr(out_ids), _ptr(out_d2), _stream(stream)))
        return out_ids, out_d2

    def knn_stats(self, q: torch.Tensor, k: int, stream=None):
        """k-NN with traversal counters: (ids, d2, {nodes, leaves, points, queries, children})."""
        q = q.contiguous()
        nq = int(q.shape[0])
        out_ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        out_d2 = torch.empty((nq, k), dtype=torch.int64, device=q.device)
        st = torch.zeros(5, dtype=torch.int64, device=q.device)
        _check(lib().psi_knn_instrumented(self._h, _ptr(q), nq, k, _ptr(out_ids), _ptr(out_d2), _ptr(st),
                                          _stream(stream)))
        c = st.cpu().tolist()
        return out_ids, out_d2, {"nodes": c[0], "leaves": c[1], "points": c[2], "queries": c[3], "children": c[4]}

    def range_count(self, boxes: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        boxes = boxes.contiguous()
        nq = int(boxes.shape[0])
        if out is None:
            out = torch.empty(nq, dtype=torch.int64, device=boxes.device)
        _check(lib().psi_range_count(self._h, _ptr(boxes), nq, _ptr(out), _stream(stream)))
        return out

    def range_report(self, boxes: torch.Tensor, capacity: int | None = None, sort: bool = False, stream=None):
        """(offsets[q+1], ids[total]); grows the output once if capacity is too small.  Without a
        capacity the output is sized from the ids per box of this index's earlier calls."""
        boxes = boxes.contiguous()
        nq = int(boxes.shape[0])
        off = torch.empty(nq + 1, dtype=torch.int64, device=boxes.device)
        cap = capacity if capacity is not None else max(1024, int(nq * self._ids_per_box * 1.25) + 1024)
        total = ctypes.c_int64(0)
        for _ in range(2):
            ids = torch.empty(max(cap, 1), dtype=torch.int32, device=boxes.device)
            st = lib().psi_range_report(self._h, _ptr(boxes), nq, _ptr(off), _ptr(ids), cap, ctypes.byref(total),
                                        REPORT_SORTED if sort else 0, _stream(stream))
            if st == ERR_CAPACITY:
                cap = int(total.value)
                continue
            _check(st)
            if nq:
                self._ids_per_box = max(1.0, 0.5 * self._ids_per_box + 0.5 * total.value / nq)
            return off, ids[:total.value]
        _check(st)

    # ---- inspection ----
    def leaves(self, stream=None):
        L, D = self.num_leaves, self.dim
        dev = torch.device("cuda", torch.cuda.current_device())
        cnt = torch.empty(L, dtype=torch.int32, device=dev)
        lo = torch.empty((L, D), dtype=torch.int32, device=dev)
        hi = torch.empty((L, D), dtype=torch.int32, device=dev)
        sk = torch.empty(L, dtype=torch.int64, device=dev)
        si = torch.empty(L, dtype=torch.int32, device=dev)
        if L:
            _check(lib().psi_export_leaves(self._h, _ptr(cnt), _ptr(lo), _ptr(hi), _ptr(sk), _ptr(si),
                                           _stream(stream)))
        return {"count": cnt, "lo": lo, "hi": hi, "sep_key": sk, "sep_id": si}

    def points(self, stream=None):
        n, D = len(self), self.dim
        dev = torch.device("cuda", torch.cuda.current_device())
        pts = torch.empty((n, D), dtype=torch.int32, device=dev)
        ids = torch.empty(n, dtype=torch.int32, device=dev)
        keys = torch.empty(n, dtype=torch.int64, device=dev)
        leaf = torch.empty(n, dtype=torch.int32, device=dev)
        if n:
            _check(lib().psi_export_points(self._h, _ptr(pts), _ptr(ids), _ptr(keys), _ptr(leaf), _stream(stream)))
        return {"pts": pts, "ids": ids, "keys": keys, "leaf": leaf}

    def nodes(self, stream=None):
        N, D = self.num_nodes, self.dim
        dev = torch.device("cuda", torch.cuda.current_device())
        depth = torch.empty(N, dtype=torch.int32, device=dev)
        prefix = torch.empty(N, dtype=torch.int64, device=dev)
        cnt = torch.empty(N, dtype=torch.int64, device=dev)
        lo = torch.empty((N, D), dtype=torch.int32, device=dev)
        hi = torch.empty((N, D), dtype=torch.int32, device=dev)
        leaf = torch.empty(N, dtype=torch.int32, device=dev)
        if N:
            _check(lib().psi_export_nodes(self._h, _ptr(depth), _ptr(prefix), _ptr(cnt), _ptr(lo), _ptr(hi),
                                          _ptr(leaf), _stream(stream)))
        return {"depth": depth, "prefix": prefix, "count": cnt, "lo": lo, "hi": hi, "is_leaf": leaf}


class Batch:
    """Many independent SPaC indexes over one concatenated point array, built in
    one persistent launch (psi_batch_*)."""

    def __init__(self, offsets, *, dim: int = 2, kind: int | str = SPAC_H, leaf_size: int = 32,
                 coord_bits: int | None = None, fanout: int = 32, threads: int = 0, radix_bits: int = 0,
                 stream=None):
        import numpy as np
        if isinstance(kind, str):
            kind = KINDS[kind]
        coord_bits = coord_bits or (30 if dim == 2 else 21)
        self.dim, self.nidx = dim, len(offsets) - 1
        self.cfg = Config(dim, kind, leaf_size, coord_bits, fanout, radix_bits)
        self._off = np.ascontiguousarray(offsets, dtype=np.int64)
        h = ctypes.c_void_p()
        _check(lib().psi_batch_create(ctypes.byref(self.cfg), self._off.ctypes.data_as(ctypes.c_void_p), self.nidx,
                                      threads, _stream(stream), ctypes.byref(h)))
        self._h = h
        self._qcap = 0

    def build(self, pts: torch.Tensor, ids: torch.Tensor, stream=None):
        _check(lib().psi_batch_build(self._h, _ptr(pts.contiguous()), _ptr(_u32(ids).contiguous()), _stream(stream)))

    def reserve(self, max_queries: int, stream=None):
        _check(lib().psi_batch_knn_reserve(self._h, int(max_queries), _stream(stream)))
        self._qcap = max(self._qcap, int(max_queries))

    def knn(self, q: torch.Tensor, qoffsets: torch.Tensor, k: int, out_ids=None, out_d2=None, stream=None):
        nq = int(q.shape[0])
        if nq > self._qcap:
            self.reserve(nq, stream)
        if out_ids is None:
            out_ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        if out_d2 is None:
            out_d2 = torch.empty((nq, k), dtype=torch.int64, device=q.device)
        _check(lib().psi_batch_knn(self._h, _ptr(q.contiguous()), _ptr(qoffsets.contiguous()), nq, k, _ptr(out_ids),
                                   _ptr(out_d2), _stream(stream)))
        return out_ids, out_d2

    def knn_stats(self, q: torch.Tensor, qoffsets: torch.Tensor, k: int, stream=None):
        """Batched k-NN with traversal counters: (ids, d2, {nodes, leaves, points, queries, children})."""
        nq = int(q.shape[0])
        if nq > self._qcap:
            self.reserve(nq, stream)
        out_ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        out_d2 = torch.empty((nq, k), dtype=torch.int64, device=q.device)
        st = torch.zeros(5, dtype=torch.int64, device=q.device)
        _check(lib().psi_batch_knn_instrumented(self._h, _ptr(q.contiguous()), _ptr(qoffsets.contiguous()), nq, k,
                                                _ptr(out_ids), _ptr(out_d2), _ptr(st), _stream(stream)))
        c = st.cpu().tolist()
        return out_ids, out_d2, {"nodes": c[0], "leaves": c[1], "points": c[2], "queries": c[3], "children": c[4]}

    def sync(self, stream=None):
        _check(lib().psi_batch_sync(self._h, _stream(stream)))

    def leaves(self, i: int, stream=None):
        L = int(lib().psi_batch_num_leaves(self._h, i))
        dev = torch.device("cuda", torch.cuda.current_device())
        cnt = torch.empty(L, dtype=torch.int32, device=dev)
        lo = torch.empty((L, self.dim), dtype=torch.int32, device=dev)
        hi = torch.empty((L, self.dim), dtype=torch.int32, device=dev)
        n = ctypes.c_int64(0)
        if L:
            _check(lib().psi_batch_export_index(self._h, i, _ptr(cnt), _ptr(lo), _ptr(hi), ctypes.byref(n),
                                                _stream(stream)))
        return {"count": cnt, "lo": lo, "hi": hi}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().psi_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FConfig(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("leaf_size", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("lo", ctypes.c_float * 8), ("hi", ctypes.c_float * 8)]


class FOrth:
    """P-Orth over float32 coordinates in D = 2..5, built by midpoint splits of the region [lo, hi)^D."""

    def __init__(self, pts: torch.Tensor, ids: torch.Tensor, lo, hi, *, leaf_size: int = 32, max_depth: int = 48,
                 stream=None):
        pts = pts.contiguous()
        self.dim = int(pts.shape[1])
        self.cfg = FConfig(self.dim, leaf_size, max_depth)
        for d in range(self.dim):
            self.cfg.lo[d] = float(lo[d])
            self.cfg.hi[d] = float(hi[d])
        h = ctypes.c_void_p()
        ids = _u32(ids).contiguous()
        _check(lib().psi_forth_build(ctypes.byref(self.cfg), _ptr(pts), _ptr(ids), int(pts.shape[0]),
                                     _stream(stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().psi_forth_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self) -> int:
        return int(lib().psi_forth_size(self._h))

    @property
    def num_nodes(self) -> int:
        return int(lib().psi_forth_num_nodes(self._h))

    def sync(self, stream=None):
        _check(lib().psi_forth_sync(self._h, _stream(stream)))

    def insert(self, pts: torch.Tensor, ids: torch.Tensor, stream=None):
        _check(lib().psi_forth_insert(self._h, _ptr(pts.contiguous()), _ptr(_u32(ids).contiguous()),
                                      int(pts.shape[0]), _stream(stream)))

    def delete(self, pts: torch.Tensor, ids: torch.Tensor, num_deleted: torch.Tensor | None = None, stream=None):
        _check(lib().psi_forth_delete(self._h, _ptr(pts.contiguous()), _ptr(_u32(ids).contiguous()),
                                      int(pts.shape[0]), _ptr(num_deleted), _stream(stream)))

    def knn(self, q: torch.Tensor, k: int, stream=None):
        q = q.contiguous()
        nq = int(q.shape[0])
        out_ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        out_d2 = torch.empty((nq, k), dtype=torch.float64, device=q.device)
        _check(lib().psi_forth_knn(self._h, _ptr(q), nq, k, _ptr(out_ids), _ptr(out_d2), _stream(stream)))
        return out_ids, out_d2

    def range_count(self, boxes: torch.Tensor, stream=None):
        boxes = boxes.contiguous()
        nq = int(boxes.shape[0])
        out = torch.empty(nq, dtype=torch.int64, device=boxes.device)
        _check(lib().psi_forth_range_count(self._h, _ptr(boxes), nq, _ptr(out), _stream(stream)))
        return out

    def nodes(self, stream=None):
        N, n, D = self.num_nodes, len(self), self.dim
        dev = torch.device("cuda", torch.cuda.current_device())
        out = {"depth": torch.empty(N, dtype=torch.int32, device=dev), "count": torch.empty(N, dtype=torch.int32, device=dev),
               "kids": torch.empty(N, dtype=torch.int32, device=dev), "ref": torch.empty(N, dtype=torch.int32, device=dev),
               "lo": torch.empty((N, D), dtype=torch.float32, device=dev),
               "hi": torch.empty((N, D), dtype=torch.float32, device=dev),
               "pts": torch.empty((n, D), dtype=torch.float32, device=dev),
               "ids": torch.empty(n, dtype=torch.int32, device=dev)}
        if N or n:
            _check(lib().psi_forth_export(self._h, *(_ptr(out[k]) for k in ("depth", "count", "kids", "ref", "lo", "hi",
                                                                              "pts", "ids")), _stream(stream)))
        return out


def encode(pts: torch.Tensor, kind: int | str = SPAC_Z, coord_bits: int | None = None, stream=None) -> torch.Tensor:
    if isinstance(kind, str):
        kind = KINDS[kind]
    dim = int(pts.shape[1])
    coord_bits = coord_bits or (30 if dim == 2 else 21)
    cfg = Config(dim, kind, 32, coord_bits, 32, 0)
    pts = pts.contiguous()
    keys = torch.empty(pts.shape[0], dtype=torch.int64, device=pts.device)
    _check(lib().psi_encode(ctypes.byref(cfg), _ptr(pts), int(pts.shape[0]), _ptr(keys), _stream(stream)))
    return keys


def sort_pairs(keys: torch.Tensor, vals: torch.Tensor, key_bits: int = 64, stream=None):
    """In-place stable sort of (uint64 key, uint32 value) pairs by key."""
    _check(lib().psi_sort_pairs(_ptr(keys), _ptr(vals), int(keys.shape[0]), key_bits, _stream(stream)))
    return keys, vals


def test_sort_withheld_tile(keys: torch.Tensor, vals: torch.Tensor, withheld_tile: int, spin_limit: int,
                            stream=None) -> int:
    """Test hook of the bounded look-back waits: returns the library status
    (OK, or ERR_DEVICE_TIMEOUT when the withheld tile made a wait run out)."""
    return int(lib().psi_test_sort_withheld_tile(_ptr(keys), _ptr(vals), int(keys.shape[0]), int(withheld_tile),
                                                 int(spin_limit), _stream(stream)))


def launch_count() -> int:
    return int(lib().psi_launch_count())


def profile_enable(on: bool = True):
    lib().psi_profile_enable(1 if on else 0)


def profile_reset():
    lib().psi_profile_reset()


def profile_read(name: str):
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0)
    lib().psi_profile_read(name.encode(), ctypes.byref(n), ctypes.byref(ms))
    return int(n.value), float(ms.value)


def profile_dump() -> dict:
    size = lib().psi_profile_dump(None, 0)
    buf = ctypes.create_string_buffer(size + 1)
    lib().psi_profile_dump(buf, size + 1)
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.rsplit(" ", 2)
        out[name] = (int(cnt), float(ms))
    return out
