"""Parity at the benchmark's full size (1e8 2D clustered points, SPaC-H, leaf
size 32, the same calls bench.py times): sampled k-NN answers and range counts
against the oracle's definitions over the raw point arrays, plus structural
properties that hold at any size."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2601_05347_gb300 import gen  # noqa: E402

pytestmark = pytest.mark.gpu


def test_full_size_build_update_query_sampled():
    from paper_2601_05347_gb300 import psi
    n = 100_000_000
    dev = "cuda"
    pts = gen.varden(n, 2, 30, gen.config_seed(1, 0), x_range=(0, 1 << 29))
    ids = np.arange(n, dtype=np.uint32)
    ins = gen.varden(1_000_000, 2, 30, gen.config_seed(1, 1), x_range=(0, 1 << 29))
    ins_ids = np.arange(n, n + 1_000_000, dtype=np.uint32)
    dsel = gen.sample_without_replacement(n, 1_000_000, gen.config_seed(1, 2))
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32) if a.dtype == np.uint32 else a).to(dev)
    ix = psi.Index(T(pts), T(ids), kind="spac_h", leaf_size=32)
    ix.insert(T(ins), T(ins_ids))
    nd = torch.zeros(1, dtype=torch.int64, device=dev)
    ix.delete(T(pts[dsel]), T(ids[dsel]), nd)
    ix.sync()
    assert int(nd.item()) == 1_000_000
    assert len(ix) == n
    # structure at any size: counts add up, every leaf within 1..2*phi
    lv = ix.leaves()
    cnt = lv["count"].cpu().numpy()
    assert int(cnt.sum()) == n and cnt.min() >= 1 and cnt.max() <= 64
    # the live set, for the sampled checks
    keep = np.ones(n, bool)
    keep[dsel] = False
    live_p = np.concatenate([pts[keep], ins])
    live_i = np.concatenate([ids[keep], ins_ids])
    # 1e7 queries as in the benchmark; 6 sampled answers checked one by one
    q = pts[gen.sample_with_replacement(n, 10_000_000, gen.config_seed(1, 3))]
    gi, gd = ix.knn(T(q), 10)
    sample = gen.sample_with_replacement(len(q), 6, 12345)
    oi, od = O.knn_brute_raw(live_p, live_i, q[sample], 10)
    assert (gi[T(sample)].cpu().numpy().view(np.uint32) == oi).all()
    assert (gd[T(sample)].cpu().numpy() == od).all()
    boxes = gen.centred_boxes(pts[gen.sample_with_replacement(n, 50_000, 7)], 8643, 30)
    gc = ix.range_count(T(boxes)).cpu().numpy()
    bs = gen.sample_with_replacement(len(boxes), 6, 99)
    assert (gc[bs] == O.range_count_brute_raw(live_p, boxes[bs])).all()
    off, rid = ix.range_report(T(boxes))
    off = off.cpu().numpy()
    assert (np.diff(off) == gc).all()
    ix.close()
