"""Failure detection without a GPU fault: a digit pass whose tile withholds its
look-back words makes the waiting tiles give up after a short, bounded number
of polls; the call reports PSI_ERR_DEVICE_TIMEOUT, and the same process then
sorts correctly (the context stays usable)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2601_05347_gb300 import gen  # noqa: E402

pytestmark = pytest.mark.gpu

TILE = 4096


def _pairs(n, seed):
    k = gen.splitmix64(seed, np.arange(n, dtype=np.uint64))
    v = np.arange(n, dtype=np.uint32)
    return k, v


def _dev(k, v):
    return torch.from_numpy(k.view(np.int64)).cuda(), torch.from_numpy(v.view(np.int32)).cuda()


def test_withheld_look_back_word_times_out_then_sorts_again():
    from paper_2601_05347_gb300 import psi
    n = 5 * TILE + 123
    k, v = _pairs(n, 3)
    order = np.argsort(k, kind="stable")
    # no tile withheld: the hook is an ordinary sort
    dk, dv = _dev(k, v)
    assert psi.test_sort_withheld_tile(dk, dv, -1, 1 << 10) == psi.OK
    assert (dk.cpu().numpy().view(np.uint64) == k[order]).all()
    assert (dv.cpu().numpy().view(np.uint32) == v[order]).all()
    # tile 1 never publishes: tile 2 (at least) waits 2^10 polls and gives up
    dk, dv = _dev(k, v)
    assert psi.test_sort_withheld_tile(dk, dv, 1, 1 << 10) == psi.ERR_DEVICE_TIMEOUT
    assert "timed out" in psi.lib().psi_last_error().decode()
    # the context is still usable: the library's sort and the hook sort correctly
    dk, dv = _dev(k, v)
    psi.sort_pairs(dk, dv, 64)
    torch.cuda.synchronize()
    assert (dk.cpu().numpy().view(np.uint64) == k[order]).all()
    assert (dv.cpu().numpy().view(np.uint32) == v[order]).all()
    dk, dv = _dev(k, v)
    assert psi.test_sort_withheld_tile(dk, dv, -1, 1 << 10) == psi.OK
    assert (dk.cpu().numpy().view(np.uint64) == k[order]).all()


def test_withheld_last_tile_has_no_waiter():
    # the last tile has no successor, so nothing waits on it: the sort is exact
    from paper_2601_05347_gb300 import psi
    n = 3 * TILE + 7
    k, v = _pairs(n, 5)
    order = np.argsort(k, kind="stable")
    dk, dv = _dev(k, v)
    assert psi.test_sort_withheld_tile(dk, dv, 3, 1 << 10) == psi.OK
    assert (dk.cpu().numpy().view(np.uint64) == k[order]).all()
    assert (dv.cpu().numpy().view(np.uint32) == v[order]).all()
