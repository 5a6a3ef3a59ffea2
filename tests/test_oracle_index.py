"""Pins of the oracle's index and queries: brute force on tiny inputs written
independently with numpy, hand-checked examples, and the structural invariants
the paper fixes (Algorithm 3 leaf wrapping, tight boxes, counts)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2601_05347_gb300 import gen


def np_knn(pts, ids, q, k):
    """k-NN by definition: sort all points by (squared distance, id)."""
    out_i = np.full((len(q), k), 0xFFFFFFFF, np.uint32)
    out_d = np.full((len(q), k), np.iinfo(np.int64).max, np.int64)
    P = pts.astype(np.int64)
    for t, qq in enumerate(q.astype(np.int64)):
        d2 = ((P - qq) ** 2).sum(axis=1)
        order = np.lexsort((ids, d2))[:k]
        out_i[t, :len(order)] = ids[order]
        out_d[t, :len(order)] = d2[order]
    return out_i, out_d


def np_inbox(pts, box):
    D = pts.shape[1]
    return np.all((pts >= box[:D]) & (pts <= box[D:]), axis=1)


def make(n, dim=2, bits=30, seed=0, dup=False, kind=O.SPAC_Z, phi=8, fanout=4):
    rng = np.random.default_rng(seed)
    hi = min(1 << bits, 64 if dup else 1 << bits)
    pts = rng.integers(0, hi, size=(n, dim)).astype(np.int32)
    ids = rng.permutation(n).astype(np.uint32) * 3 + 5
    return pts, ids, O.Index(pts, ids, dim=dim, kind=kind, phi=phi, bits=bits, fanout=fanout)


def test_knn_worked_example():
    # points on a line; the query at x=2 is equidistant from x=1 and x=3
    pts = np.array([[0, 0], [1, 0], [3, 0], [10, 0]], np.int32)
    ids = np.array([7, 9, 4, 1], np.uint32)
    ix = O.Index(pts, ids, phi=2, fanout=2)
    i, d = ix.knn(np.array([[2, 0]]), 3)
    assert i.tolist() == [[4, 9, 7]]  # d2 = 1 (id 4), 1 (id 9), 4 (id 7)
    assert d.tolist() == [[1, 1, 4]]
    i, d = ix.knn(np.array([[2, 0]]), 6)  # k > n pads
    assert i[0, 4:].tolist() == [0xFFFFFFFF] * 2 and d[0, 4] == np.iinfo(np.int64).max


@pytest.mark.parametrize("dim,bits,kind", [(2, 30, O.SPAC_Z), (2, 30, O.SPAC_H), (3, 21, O.SPAC_Z), (2, 8, O.PORTH)])
@pytest.mark.parametrize("dup", [False, True])
def test_knn_matches_brute_force(dim, bits, kind, dup):
    pts, ids, ix = make(700, dim, bits, seed=dim + bits, dup=dup, kind=kind)
    rng = np.random.default_rng(3)
    q = rng.integers(0, min(1 << bits, 80 if dup else 1 << bits), size=(60, dim)).astype(np.int32)
    q[:10] = pts[:10]  # queries on data points
    for k in (1, 5, 32, 700, 710):
        gi, gd = ix.knn(q, k)
        bi, bd = ix.knn(q, k, brute=True)
        ni, nd = np_knn(pts, ids, q, k)
        assert (gi == ni).all() and (gd == nd).all()
        assert (bi == ni).all() and (bd == nd).all()


def test_knn_empty_index():
    ix = O.Index(np.zeros((0, 2), np.int32), np.zeros(0, np.uint32))
    i, d = ix.knn(np.array([[1, 2]]), 3)
    assert (i == 0xFFFFFFFF).all() and (d == np.iinfo(np.int64).max).all()
    assert ix.range_count(np.array([[0, 0, 10, 10]])).tolist() == [0]


@pytest.mark.parametrize("dim,bits", [(2, 30), (3, 21), (2, 6)])
def test_range_matches_brute_force(dim, bits):
    pts, ids, ix = make(900, dim, bits, seed=11, dup=bits == 6)
    rng = np.random.default_rng(4)
    lo = rng.integers(0, 1 << bits, size=(80, dim))
    side = rng.integers(0, 1 << (bits - 1), size=(80, dim))
    boxes = np.concatenate([lo, np.minimum(lo + side, (1 << bits) - 1)], axis=1).astype(np.int32)
    boxes[0] = [0] * dim + [(1 << bits) - 1] * dim          # everything
    boxes[1] = list(pts[3]) + list(pts[3])                  # a degenerate box on a point
    boxes[2] = [5] * dim + [4] * dim                        # lo > hi: empty
    c = ix.range_count(boxes)
    cb = ix.range_count(boxes, brute=True)
    off, rid = ix.range_report(boxes)
    for t, b in enumerate(boxes):
        m = np_inbox(pts, b)
        assert c[t] == m.sum() == cb[t]
        assert sorted(ids[m].tolist()) == rid[off[t]:off[t + 1]].tolist()
    assert c[0] == 900 and c[2] == 0 and c[1] >= 1


def test_range_closed_boundaries():
    pts = np.array([[10, 10], [20, 20], [15, 25]], np.int32)
    ix = O.Index(pts, np.arange(3, dtype=np.uint32), phi=1, fanout=2)
    assert ix.range_count(np.array([[10, 10, 20, 20]])).tolist() == [2]
    assert ix.range_count(np.array([[11, 10, 20, 19]])).tolist() == [0]
    assert ix.range_count(np.array([[15, 25, 15, 25]])).tolist() == [1]


@pytest.mark.parametrize("kind", [O.SPAC_Z, O.SPAC_H])
def test_layout_invariants(kind):
    pts, ids, ix = make(1000, 2, 30, seed=2, kind=kind, phi=16, fanout=8)
    keys, sid, spts = ix.points()
    # sorted by (key, id), the key being the curve key of the point
    assert sorted(zip(keys.tolist(), sid.tolist())) == list(zip(keys.tolist(), sid.tolist()))
    assert (keys == O.keys(spts, 2, kind, 30)).all()
    # point multiset preserved
    assert sorted(zip(ids.tolist(), map(tuple, pts.tolist()))) == sorted(zip(sid.tolist(), map(tuple, spts.tolist())))
    lv = ix.levels()
    L = -(-1000 // 16)
    assert len(lv[0]["count"]) == L and lv[-1]["count"].tolist() == [1000]
    for i in range(L):
        seg = spts[i * 16:(i + 1) * 16]
        assert lv[0]["count"][i] == len(seg)
        assert (lv[0]["lo"][i] == seg.min(0)).all() and (lv[0]["hi"][i] == seg.max(0)).all()
        assert lv[0]["first_key"][i] == keys[i * 16] and lv[0]["first_id"][i] == sid[i * 16]
    for l in range(1, len(lv)):
        ch = lv[l - 1]
        for j in range(len(lv[l]["count"])):
            s = slice(j * 8, (j + 1) * 8)
            assert lv[l]["count"][j] == ch["count"][s].sum()
            assert (lv[l]["lo"][j] == ch["lo"][s].min(0)).all() and (lv[l]["hi"][j] == ch["hi"][s].max(0)).all()


def test_duplicate_keys_ordered_by_id():
    pts = np.array([[5, 5]] * 6 + [[1, 1]] * 3, np.int32)
    ids = np.array([9, 3, 7, 1, 8, 2, 6, 5, 4], np.uint32)
    ix = O.Index(pts, ids, phi=4, fanout=2)
    k, i, p = ix.points()
    assert i.tolist() == [4, 5, 6, 1, 2, 3, 7, 8, 9]


def test_updates_point_set():
    pts, ids, ix = make(500, 2, 30, seed=5, phi=8)
    rng = np.random.default_rng(8)
    new = rng.integers(0, 1 << 30, size=(200, 2)).astype(np.int32)
    nid = np.arange(10000, 10200, dtype=np.uint32)
    ix.insert(new, nid)
    allp = np.concatenate([pts, new])
    alli = np.concatenate([ids, nid])
    assert len(ix) == 700
    sel = rng.permutation(700)[:300]
    dp, di = allp[sel], alli[sel]
    # an absent pair (right id, wrong point) and a duplicate request are ignored
    dp = np.concatenate([dp, [[1, 2]], dp[:1]])
    di = np.concatenate([di, di[1:2], di[:1]])
    assert ix.delete(dp, di) == 300
    keep = np.ones(700, bool)
    keep[sel] = False
    k, i, p = ix.points()
    assert sorted(zip(i.tolist(), map(tuple, p.tolist()))) == sorted(zip(alli[keep].tolist(), map(tuple, allp[keep].tolist())))
    q = rng.integers(0, 1 << 30, size=(30, 2)).astype(np.int32)
    gi, gd = ix.knn(q, 7)
    ni, nd = np_knn(allp[keep], alli[keep], q, 7)
    assert (gi == ni).all() and (gd == nd).all()
    # layout after the update equals a fresh build of the same set
    fresh = O.Index(allp[keep], alli[keep], phi=8, fanout=4)
    for a, b in zip(ix.levels(), fresh.levels()):
        for key in a:
            assert (a[key] == b[key]).all()


def test_generator_workload_runs():
    p = gen.varden(3000, 2, 30, 1)
    ix = O.Index(p, np.arange(3000, dtype=np.uint32), kind=O.SPAC_H, phi=32)
    i, d = ix.knn(p[:20], 10)
    ni, nd = np_knn(p, np.arange(3000, dtype=np.uint32), p[:20], 10)
    assert (i == ni).all() and (d == nd).all()


def test_raw_brute_force_matches_numpy():
    rng = np.random.default_rng(12)
    pts = rng.integers(0, 1 << 30, size=(800, 2)).astype(np.int32)
    ids = (rng.permutation(800) * 7 + 1).astype(np.uint32)
    q = rng.integers(0, 1 << 30, size=(20, 2)).astype(np.int32)
    oi, od = O.knn_brute_raw(pts, ids, q, 9)
    ni, nd = np_knn(pts, ids, q, 9)
    assert (oi == ni).all() and (od == nd).all()
    boxes = np.concatenate([q, q + (1 << 27)], axis=1).astype(np.int32)
    c = O.range_count_brute_raw(pts, boxes)
    assert c.tolist() == [int(np_inbox(pts, b).sum()) for b in boxes]
