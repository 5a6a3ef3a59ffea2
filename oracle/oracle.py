"""ctypes wrapper over the C oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.

The oracle is a plain sequential CPU restatement of the operations of "Parallel
Dynamic Spatial Indexes" (PPoPP '26, arXiv 2601.05347).  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "psi_oracle.c")
SRC_F = os.path.join(HERE, "psi_oracle_f.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

SPAC_Z, SPAC_H, PORTH = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C11, no target-specific flags)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    stale = not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
        os.path.getmtime(SRC), os.path.getmtime(SRC_F), os.path.getmtime(os.path.join(HERE, "psi_oracle.h")))
    if force or stale:
        tmp = LIB + f".tmp{os.getpid()}"
        # -ffp-contract=off: every float/double operation rounds on its own (no fused multiply-add)
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", SRC, SRC_F, "-lm",
                               "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


class _Cfg(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("kind", ctypes.c_int), ("phi", ctypes.c_int),
                ("bits", ctypes.c_int), ("fanout", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.or_morton.restype = ctypes.c_uint64
        L.or_morton.argtypes = [P, ctypes.c_int, ctypes.c_int]
        L.or_hilbert2.restype = ctypes.c_uint64
        L.or_hilbert2.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int]
        L.or_hilbert3.restype = ctypes.c_uint64
        L.or_hilbert3.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int]
        L.or_keys.restype = ctypes.c_int
        L.or_keys.argtypes = [P, P, i64, P]
        L.or_build.restype = P
        L.or_build.argtypes = [P, P, P, i64]
        L.or_free.argtypes = [P]
        L.or_size.restype = i64
        L.or_size.argtypes = [P]
        L.or_insert.argtypes = [P, P, P, i64]
        L.or_delete.restype = i64
        L.or_delete.argtypes = [P, P, P, i64]
        L.or_points.argtypes = [P, P, P, P]
        L.or_num_levels.restype = ctypes.c_int
        L.or_num_levels.argtypes = [P]
        L.or_level_size.restype = i64
        L.or_level_size.argtypes = [P, ctypes.c_int]
        L.or_level.argtypes = [P, ctypes.c_int, P, P, P, P, P]
        for f in (L.or_knn, L.or_knn_brute):
            f.argtypes = [P, P, i64, ctypes.c_int, P, P]
        for f in (L.or_range_count, L.or_range_count_brute):
            f.argtypes = [P, P, i64, P]
        L.or_range_report.restype = i64
        L.or_range_report.argtypes = [P, P, i64, P, P, i64]
        L.or_knn_brute_raw.argtypes = [P, P, i64, ctypes.c_int, P, i64, ctypes.c_int, P, P]
        L.or_forth_build.restype = P
        L.or_forth_build.argtypes = [P, P, P, i64]
        L.or_forth_free.argtypes = [P]
        L.or_forth_num_nodes.restype = i64
        L.or_forth_num_nodes.argtypes = [P]
        L.or_forth_export.argtypes = [P, P, P, P, P, P, P, P, P]
        L.or_fknn_brute.argtypes = [P, P, i64, ctypes.c_int, P, i64, ctypes.c_int, P, P]
        L.or_frange_count_brute.argtypes = [P, i64, ctypes.c_int, P, i64, P]
        L.or_range_count_brute_raw.argtypes = [P, i64, ctypes.c_int, P, i64, P]
        L.or_porth.restype = i64
        L.or_porth.argtypes = [P, i64, P, P, P, P, P, P]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def morton(p, dim: int, bits: int) -> int:
    a = _c(p, np.int32)
    return int(lib().or_morton(_ptr(a), dim, bits))


def hilbert2(x: int, y: int, bits: int) -> int:
    return int(lib().or_hilbert2(int(x), int(y), bits))


def hilbert3(x: int, y: int, z: int, bits: int) -> int:
    return int(lib().or_hilbert3(int(x), int(y), int(z), bits))


def keys(pts, dim: int, kind: int, bits: int) -> np.ndarray:
    pts = _c(pts, np.int32).reshape(-1, dim)
    out = np.empty(len(pts), np.uint64)
    cfg = _Cfg(dim, kind, 32, bits, 32)
    if lib().or_keys(ctypes.byref(cfg), _ptr(pts), len(pts), _ptr(out)) != 0:
        raise ValueError("coordinate outside [0, 2^bits)")
    return out


def knn_brute_raw(pts, ids, q, k):
    """k-NN by definition over raw arrays (no index)."""
    pts = _c(pts, np.int32)
    dim = pts.shape[1]
    ids = _c(ids, np.uint32)
    q = _c(q, np.int32).reshape(-1, dim)
    oi = np.empty((len(q), k), np.uint32)
    od = np.empty((len(q), k), np.int64)
    lib().or_knn_brute_raw(_ptr(pts), _ptr(ids), len(pts), dim, _ptr(q), len(q), k, _ptr(oi), _ptr(od))
    return oi, od


def range_count_brute_raw(pts, boxes):
    pts = _c(pts, np.int32)
    dim = pts.shape[1]
    boxes = _c(boxes, np.int32).reshape(-1, 2 * dim)
    out = np.empty(len(boxes), np.int64)
    lib().or_range_count_brute_raw(_ptr(pts), len(pts), dim, _ptr(boxes), len(boxes), _ptr(out))
    return out


class Index:
    """The oracle's sorted-key index (see psi_oracle.c)."""

    def __init__(self, pts, ids, *, dim=2, kind=SPAC_Z, phi=32, bits=30, fanout=32):
        self.dim, self.kind, self.phi, self.bits, self.fanout = dim, kind, phi, bits, fanout
        self._cfg = _Cfg(dim, kind, phi, bits, fanout)
        pts = _c(pts, np.int32).reshape(-1, dim)
        ids = _c(ids, np.uint32)
        assert len(pts) == len(ids)
        h = lib().or_build(ctypes.byref(self._cfg), _ptr(pts), _ptr(ids), len(pts))
        if not h:
            raise ValueError("coordinate outside [0, 2^bits)")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_free(h)
            self._h = None

    def __len__(self):
        return int(lib().or_size(self._h))

    def insert(self, pts, ids):
        pts = _c(pts, np.int32).reshape(-1, self.dim)
        ids = _c(ids, np.uint32)
        lib().or_insert(self._h, _ptr(pts), _ptr(ids), len(pts))

    def delete(self, pts, ids) -> int:
        pts = _c(pts, np.int32).reshape(-1, self.dim)
        ids = _c(ids, np.uint32)
        return int(lib().or_delete(self._h, _ptr(pts), _ptr(ids), len(pts)))

    def points(self):
        """(keys, ids, pts) of the live points in (key, id) order."""
        n = len(self)
        k = np.empty(n, np.uint64)
        i = np.empty(n, np.uint32)
        p = np.empty((n, self.dim), np.int32)
        lib().or_points(self._h, _ptr(k), _ptr(i), _ptr(p))
        return k, i, p

    def levels(self):
        """Summary tree, leaves first: list of dicts with lo, hi, count (+ first_key, first_id at level 0)."""
        out = []
        for l in range(lib().or_num_levels(self._h)):
            S = int(lib().or_level_size(self._h, l))
            lo = np.empty((S, self.dim), np.int32)
            hi = np.empty((S, self.dim), np.int32)
            cnt = np.empty(S, np.int64)
            fk = np.empty(S, np.uint64)
            fi = np.empty(S, np.uint32)
            lib().or_level(self._h, l, _ptr(lo), _ptr(hi), _ptr(cnt), _ptr(fk), _ptr(fi))
            d = {"lo": lo, "hi": hi, "count": cnt}
            if l == 0:
                d["first_key"], d["first_id"] = fk, fi
            out.append(d)
        return out

    def knn(self, q, k: int, brute: bool = False):
        q = _c(q, np.int32).reshape(-1, self.dim)
        ids = np.empty((len(q), k), np.uint32)
        d2 = np.empty((len(q), k), np.int64)
        f = lib().or_knn_brute if brute else lib().or_knn
        f(self._h, _ptr(q), len(q), k, _ptr(ids), _ptr(d2))
        return ids, d2

    def range_count(self, boxes, brute: bool = False):
        boxes = _c(boxes, np.int32).reshape(-1, 2 * self.dim)
        out = np.empty(len(boxes), np.int64)
        f = lib().or_range_count_brute if brute else lib().or_range_count
        f(self._h, _ptr(boxes), len(boxes), _ptr(out))
        return out

    def range_report(self, boxes):
        """(offsets[q+1], ids) with each query's ids ascending."""
        boxes = _c(boxes, np.int32).reshape(-1, 2 * self.dim)
        off = np.empty(len(boxes) + 1, np.int64)
        total = lib().or_range_report(self._h, _ptr(boxes), len(boxes), _ptr(off), None, 0)
        ids = np.empty(max(total, 1), np.uint32)
        lib().or_range_report(self._h, _ptr(boxes), len(boxes), _ptr(off), _ptr(ids), total)
        return off, ids[:total]

    def porth(self):
        """P-Orth node list in preorder: dict of depth, prefix, count, lo, hi, is_leaf."""
        n = int(lib().or_porth(self._h, 0, None, None, None, None, None, None))
        depth = np.empty(n, np.int32)
        prefix = np.empty(n, np.uint64)
        cnt = np.empty(n, np.int64)
        lo = np.empty((n, self.dim), np.int32)
        hi = np.empty((n, self.dim), np.int32)
        leaf = np.empty(n, np.int32)
        if n:
            lib().or_porth(self._h, n, _ptr(depth), _ptr(prefix), _ptr(cnt), _ptr(lo), _ptr(hi), _ptr(leaf))
        return {"depth": depth, "prefix": prefix, "count": cnt, "lo": lo, "hi": hi, "is_leaf": leaf}


# ---------------------------------------------------------------------------
# SFC-free P-Orth over float coordinates (psi_oracle_f.c)
# ---------------------------------------------------------------------------
FMAXD = 8


class _FCfg(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("phi", ctypes.c_int), ("max_depth", ctypes.c_int),
                ("lo", ctypes.c_float * FMAXD), ("hi", ctypes.c_float * FMAXD)]


def fcfg(dim, phi, lo, hi, max_depth=48):
    c = _FCfg(dim, phi, max_depth)
    for d in range(dim):
        c.lo[d] = float(lo[d])
        c.hi[d] = float(hi[d])
    return c


class FOrth:
    """The float P-Orth of a point set: node arrays in breadth-first order."""

    def __init__(self, pts, ids, lo, hi, phi=32, max_depth=48):
        self.pts = _c(pts, np.float32)
        self.dim = self.pts.shape[1]
        self.ids = _c(ids, np.uint32)
        cfg = fcfg(self.dim, phi, lo, hi, max_depth)
        h = lib().or_forth_build(ctypes.byref(cfg), _ptr(self.pts), _ptr(self.ids), len(self.pts))
        if not h:
            raise ValueError("a point lies outside the region")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_forth_free(self._h)
            self._h = None

    def nodes(self):
        n = int(lib().or_forth_num_nodes(self._h))
        D = self.dim
        out = {"depth": np.empty(n, np.int32), "count": np.empty(n, np.int64), "kids": np.empty(n, np.int32),
               "is_leaf": np.empty(n, np.int32), "lo": np.empty((n, D), np.float32),
               "hi": np.empty((n, D), np.float32), "leaf_first": np.empty(n, np.int64),
               "leaf_ids": np.empty(max(len(self.pts), 1), np.uint32)}
        if n:
            lib().or_forth_export(self._h, _ptr(out["depth"]), _ptr(out["count"]), _ptr(out["kids"]),
                                  _ptr(out["is_leaf"]), _ptr(out["lo"]), _ptr(out["hi"]), _ptr(out["leaf_first"]),
                                  _ptr(out["leaf_ids"]))
        return out

    def knn(self, q, k):
        return fknn_brute(self.pts, self.ids, q, k)

    def range_count(self, boxes):
        return frange_count_brute(self.pts, boxes)


def fknn_brute(pts, ids, q, k):
    """k-NN by definition, float points, double squared distances."""
    pts = _c(pts, np.float32)
    dim = pts.shape[1]
    ids = _c(ids, np.uint32)
    q = _c(q, np.float32).reshape(-1, dim)
    oi = np.empty((len(q), k), np.uint32)
    od = np.empty((len(q), k), np.float64)
    lib().or_fknn_brute(_ptr(pts), _ptr(ids), len(pts), dim, _ptr(q), len(q), k, _ptr(oi), _ptr(od))
    return oi, od


def frange_count_brute(pts, boxes):
    pts = _c(pts, np.float32)
    dim = pts.shape[1]
    boxes = _c(boxes, np.float32).reshape(-1, 2 * dim)
    out = np.empty(len(boxes), np.int64)
    lib().or_frange_count_brute(_ptr(pts), len(pts), dim, _ptr(boxes), len(boxes), _ptr(out))
    return out
