"""The boundary's argument checks (include/psi.h): every invalid call returns
PSI_ERR_INVALID with a message, before any CUDA call, so this runs without a
GPU.  Empty work (n = 0 sorts) returns PSI_OK without touching the device."""
import ctypes

import pytest

from paper_2601_05347_gb300 import _build, psi

INVALID, OK = 1, 0
NULL = None
P = ctypes.c_void_p(1 << 20)  # a non-null pointer that is never dereferenced: the checks fail first


@pytest.fixture(scope="module")
def L():
    _build.build()
    lib = psi.lib()
    yield lib
    # a successful call clears the message: later modules see the library as loaded fresh
    assert lib.psi_sort_pairs(NULL, NULL, 0, 60, NULL) == OK
    assert lib.psi_last_error() == b""


def cfg(dim=2, kind=psi.SPAC_Z, leaf=32, bits=30, fanout=0, radix=0):
    return psi.Config(dim, kind, leaf, bits, fanout, radix)


def build_status(L, c, n=10, pts=P, ids=P, out=True):
    h = ctypes.c_void_p()
    st = L.psi_build(ctypes.byref(c) if c is not None else NULL, pts, ids, n, NULL,
                     ctypes.byref(h) if out else NULL)
    return st, h.value


@pytest.mark.parametrize("c,why", [
    (None, "null config"), (cfg(dim=4), "dim"), (cfg(kind=7), "kind"), (cfg(leaf=0), "leaf_size"),
    (cfg(leaf=65), "leaf_size"), (cfg(bits=32), "coord_bits"), (cfg(dim=3, bits=22), "coord_bits"),
    (cfg(fanout=1), "fanout"), (cfg(fanout=33), "fanout"), (cfg(radix=9), "radix_bits")])
def test_build_rejects_bad_configs(L, c, why):
    st, h = build_status(L, c)
    assert st == INVALID and h is None
    assert why.split()[0] in L.psi_last_error().decode()


def test_build_rejects_bad_sizes_and_pointers(L):
    assert build_status(L, cfg(), out=False)[0] == INVALID
    assert build_status(L, cfg(), n=-1)[0] == INVALID
    assert build_status(L, cfg(), n=5, pts=NULL)[0] == INVALID
    assert build_status(L, cfg(), n=5, ids=NULL)[0] == INVALID
    assert build_status(L, cfg(), n=1 << 30)[0] == INVALID


def test_calls_on_a_null_index(L):
    assert L.psi_insert_batch(NULL, P, P, 3, NULL) == INVALID
    assert L.psi_delete_batch(NULL, P, P, 3, NULL, NULL) == INVALID
    assert L.psi_knn(NULL, P, 3, 10, P, P, NULL) == INVALID
    assert L.psi_range_count(NULL, P, 3, P, NULL) == INVALID
    total = ctypes.c_int64()
    assert L.psi_range_report(NULL, P, 3, P, P, 100, ctypes.byref(total), 0, NULL) == INVALID
    assert L.psi_last_error()


def test_sort_argument_checks(L):
    assert L.psi_sort_pairs(P, P, -1, 60, NULL) == INVALID
    assert L.psi_sort_pairs(P, P, 10, 0, NULL) == INVALID
    assert L.psi_sort_pairs(P, P, 10, 65, NULL) == INVALID
    assert L.psi_sort_pairs(NULL, P, 10, 60, NULL) == INVALID
    assert L.psi_sort_pairs(NULL, NULL, 0, 60, NULL) == OK  # nothing to sort
    assert L.psi_sort_pairs_noalloc(P, P, (1 << 20) + 1, 60, NULL) == INVALID
    assert "1048576" in L.psi_last_error().decode()
    assert L.psi_sort_pairs_noalloc(NULL, NULL, 0, 60, NULL) == OK


@pytest.mark.parametrize("dim,leaf,depth,lo,hi", [(1, 32, 20, 0, 1), (6, 32, 20, 0, 1), (2, 0, 20, 0, 1),
                                                  (2, 65, 20, 0, 1), (2, 32, 49, 0, 1), (2, 32, 20, 1, 1)])
def test_float_porth_rejects_bad_configs(L, dim, leaf, depth, lo, hi):
    c = psi.FConfig()
    c.dim, c.leaf_size, c.max_depth = dim, leaf, depth
    for d in range(8):
        c.lo[d], c.hi[d] = lo, hi
    h = ctypes.c_void_p()
    assert L.psi_forth_build(ctypes.byref(c), P, P, 10, NULL, ctypes.byref(h)) == INVALID
    assert h.value is None
    assert "forth" in L.psi_last_error().decode()


def test_withheld_tile_hook_rejects_bad_arguments():
    lib = ctypes.CDLL(_build.build())
    f = lib.psi_test_sort_withheld_tile
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p]
    assert f(None, None, -1, 0, 16, None) == 1          # n < 0
    assert f(None, None, 10, 0, 16, None) == 1          # null arrays
    assert f(None, None, 0, 0, 16, None) == 0           # nothing to sort


def test_batch_create_rejects_unsupported_digit_widths(L):
    off = (ctypes.c_int64 * 3)(0, 10, 20)
    h = ctypes.c_void_p()
    assert L.psi_batch_create(ctypes.byref(cfg(kind=psi.SPAC_H, radix=10)), off, 2, 0, None, ctypes.byref(h)) == INVALID
    assert b"radix_bits" in L.psi_last_error()
    assert L.psi_batch_create(ctypes.byref(cfg(kind=psi.SPAC_H, radix=11)), off, 2, 1024, None, ctypes.byref(h)) == INVALID
    assert b"11-bit" in L.psi_last_error()
