"""psi_sort_pairs_noalloc: the key sort for callers that cannot let the library
allocate device memory (a host application that owns the whole memory budget,
or a real-time loop where an allocation could stall).  Its scratch is a fixed
device array inside the library, so this test checks, through the C ABI, that
two calls in a row give exactly the allocating sort's result (integer data:
bit-exact) and that an oversized request is refused without touching the
arrays.  The file is named to run last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2601_05347_gb300 import gen  # noqa: E402

pytestmark = pytest.mark.gpu

MAX_PAIRS = 1 << 20


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _call(fn, keys, vals, bits):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(vals.data_ptr()), int(keys.shape[0]), bits, stream)


def test_noalloc_sort_matches_allocating_sort_twice():
    from paper_2601_05347_gb300 import psi
    L = psi.lib()
    # first call: the largest accepted size, many duplicate keys, 60-bit keys
    # second call: smaller and ragged (odd number of digit passes), so stale
    # histograms or look-back words from the first call would show
    for n, bits, seed in [(MAX_PAIRS, 60, 1), (300_001, 23, 2)]:
        keys = (gen.splitmix64(seed, np.arange(n, dtype=np.uint64)) >> np.uint64(64 - bits)).view(np.int64)
        keys[: n // 4] = keys[n // 4: 2 * (n // 4)]
        vals = np.arange(n, dtype=np.int32)
        ka, va = _dev(keys), _dev(vals)
        kb, vb = ka.clone(), va.clone()
        assert _call(L.psi_sort_pairs, ka, va, bits) == psi.OK
        assert _call(L.psi_sort_pairs_noalloc, kb, vb, bits) == psi.OK, L.psi_last_error()
        torch.cuda.synchronize()
        assert torch.equal(ka, kb)
        assert torch.equal(va, vb)
        order = np.argsort(keys.view(np.uint64), kind="stable")
        assert (kb.cpu().numpy() == keys[order]).all()


def test_noalloc_sort_refuses_oversized_input():
    from paper_2601_05347_gb300 import psi
    L = psi.lib()
    n = MAX_PAIRS + 1
    keys = _dev(np.arange(n, 0, -1, dtype=np.int64))
    vals = _dev(np.zeros(n, np.int32))
    before = keys.clone()
    assert _call(L.psi_sort_pairs_noalloc, keys, vals, 64) == psi.ERR_INVALID
    assert b"1048576" in L.psi_last_error()
    torch.cuda.synchronize()
    assert torch.equal(keys, before)
