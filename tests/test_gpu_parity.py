"""GPU vs oracle parity: every step of the path through the C ABI, compared
element by element with the oracle on the same seeded inputs.  All arithmetic
is integer, so the bar is bit-exact equality everywhere."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2601_05347_gb300 import gen  # noqa: E402

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2601_05347_gb300 import psi
DEV = "cuda"
KIND = {"spac_z": O.SPAC_Z, "spac_h": O.SPAC_H, "porth": O.PORTH}


def T(a):
    """numpy -> device tensor (uint32 travels as int32 bits)."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).to(DEV)


def U32(t):
    return t.cpu().numpy().view(np.uint32)


def U64(t):
    return t.cpu().numpy().view(np.uint64)


def points(n, dim, bits, seed, dup=False, clustered=False):
    if clustered:
        p = gen.varden(n, dim, bits, seed)
    else:
        p = gen.uniform(n, dim, bits, seed)
    if dup and n:
        p = (p >> (bits - 6)).astype(np.int32)  # 64 values per axis: many duplicate points
    # unique ids in shuffled order: an odd multiplier is a bijection mod 2^32
    perm = np.argsort(gen.splitmix64(seed ^ 77, np.arange(n, dtype=np.uint64)), kind="stable").astype(np.uint64)
    with np.errstate(over="ignore"):
        ids = (perm * np.uint64(2654435761) + np.uint64(12345)) & np.uint64(0xFFFFFFFF)
    return p, ids.astype(np.uint32)


# ---------------------------------------------------------------- keys, sort

@pytest.mark.parametrize("dim,bits,kind", [(2, 30, "spac_z"), (2, 30, "spac_h"), (3, 21, "spac_z"), (2, 31, "spac_h"),
                                           (2, 7, "spac_h"), (2, 1, "spac_h"), (3, 5, "porth"), (2, 31, "spac_z"),
                                           (3, 21, "spac_h"), (3, 1, "spac_h"), (3, 9, "spac_h")])
def test_encode_matches_oracle(dim, bits, kind):
    p = gen.uniform(5000, dim, bits, 3)
    p[:4] = 0
    p[4:8] = (1 << bits) - 1
    got = U64(psi.encode(T(p), kind, bits))
    want = O.keys(p, dim, KIND[kind], bits)
    assert (got == want).all()


def test_encode_rejects_out_of_range():
    p = np.array([[0, 0], [1 << 30, 5]], np.int32)
    with pytest.raises(psi.PsiError) as e:
        psi.encode(T(p), "spac_z", 30)
    assert e.value.status == psi.ERR_RANGE


@pytest.mark.parametrize("n,bits", [(1, 64), (4095, 60), (4096, 60), (4097, 60), (100003, 64), (250000, 23)])
def test_sort_pairs_is_stable_sort(n, bits):
    k = gen.splitmix64(n, np.arange(n, dtype=np.uint64)) >> np.uint64(64 - bits)
    k[: n // 3] = k[n // 3: 2 * (n // 3)]  # duplicates
    v = np.arange(n, dtype=np.uint32)
    kt, vt = T(k), T(v)
    psi.sort_pairs(kt, vt, bits)
    order = np.argsort(k, kind="stable")
    assert (U64(kt) == k[order]).all()
    assert (U32(vt) == v[order]).all()


# ---------------------------------------------------------------- build layout

def check_spac_layout(ix, o):
    lv = o.levels()
    gl = ix.leaves()
    assert ix.num_leaves == len(lv[0]["count"]) if lv else ix.num_leaves == 0
    if not lv:
        return
    assert (gl["count"].cpu().numpy() == lv[0]["count"]).all()
    assert (gl["lo"].cpu().numpy() == lv[0]["lo"]).all()
    assert (gl["hi"].cpu().numpy() == lv[0]["hi"]).all()
    assert (U64(gl["sep_key"]) == lv[0]["first_key"]).all()
    assert (U32(gl["sep_id"]) == lv[0]["first_id"]).all()
    # points: leaf by leaf the same sets as the oracle's canonical leaves
    gp = ix.points()
    gk, gi, gpts = U64(gp["keys"]), U32(gp["ids"]), gp["pts"].cpu().numpy()
    ok, oi, opts = o.points()
    leaf = gp["leaf"].cpu().numpy()
    order = np.lexsort((gi, gk, leaf))
    assert (gk[order] == ok).all() and (gi[order] == oi).all() and (gpts[order] == opts).all()
    # summary levels, stored after the leaves
    nd = ix.nodes()
    depth = nd["depth"].cpu().numpy()
    for l, want in enumerate(lv):
        sel = depth == l
        assert sel.sum() == len(want["count"])
        assert (nd["count"].cpu().numpy()[sel] == want["count"]).all()
        assert (nd["lo"].cpu().numpy()[sel] == want["lo"]).all()
        assert (nd["hi"].cpu().numpy()[sel] == want["hi"]).all()


@pytest.mark.parametrize("kind", ["spac_z", "spac_h"])
@pytest.mark.parametrize("n,phi,fanout", [(0, 32, 32), (1, 32, 32), (31, 32, 32), (32, 32, 32), (33, 32, 32),
                                          (5000, 16, 8), (100003, 32, 32), (70001, 64, 32), (20000, 1, 2)])
def test_spac_build_layout(kind, n, phi, fanout):
    p, ids = points(n, 2, 30, 11 + n, clustered=n % 2 == 1)
    ix = psi.Index(T(p), T(ids), kind=kind, leaf_size=phi, fanout=fanout)
    ix.sync()
    o = O.Index(p, ids, kind=KIND[kind], phi=phi, fanout=fanout)
    assert len(ix) == n
    check_spac_layout(ix, o)


@pytest.mark.parametrize("radix", [8, 10, 11])
@pytest.mark.parametrize("kind,dim,bits", [("spac_h", 2, 30), ("spac_z", 3, 21), ("porth", 2, 30), ("spac_h", 3, 21)])
def test_every_digit_width_gives_the_same_index(radix, kind, dim, bits):
    p, ids = points(100003, dim, bits, 61 + radix, clustered=True)
    ix = psi.Index(T(p), T(ids), kind=kind, leaf_size=32, coord_bits=bits, radix_bits=radix)
    o = O.Index(p, ids, dim=dim, kind=KIND[kind], phi=32, bits=bits)
    if kind == "porth":
        check_porth_nodes(ix, o)
    else:
        check_spac_layout(ix, o)
    newp = gen.varden(20000, dim, bits, 7 + radix)
    newi = np.arange(10_000_000, 10_020_000, dtype=np.uint32)
    ix.insert(T(newp), T(newi))
    o.insert(newp, newi)
    ix.delete(T(p[:5000]), T(ids[:5000]))
    o.delete(p[:5000], ids[:5000])
    q = query_points(2000, dim, bits, 3, p)
    gi, gd = ix.knn(T(q), 10)
    oi, od = o.knn(q, 10)
    assert (U32(gi) == oi).all() and (gd.cpu().numpy() == od).all()


@pytest.mark.parametrize("kind,dim,bits,n,clustered", [("spac_h", 2, 30, (1 << 22) + 3, True),
                                                        ("spac_z", 2, 30, (1 << 22) + 5, True),
                                                        ("porth", 3, 21, (1 << 22) + 1, True),
                                                        ("spac_h", 3, 21, (1 << 22) + 7, True),
                                                        ("spac_h", 2, 30, 1 << 22, False)])
def test_build_across_the_packed_sort_threshold(kind, dim, bits, n, clustered):
    # an encoding sort of at least 2^22 pairs whose input is locally ordered
    # (walk-ordered clustered points) packs (position, unsorted key bits) into
    # one word for its middle passes, from pass 2 at this size; its last pass
    # reads each key (Hilbert: written by the histogram pass; Morton: recomputed
    # from the point) back at its position.  Uniform input in random order
    # keeps (key, value) pairs throughout.
    p, ids = points(n, dim, bits, 71 + n % 97, clustered=clustered)
    ix = psi.Index(T(p), T(ids), kind=kind, leaf_size=32, coord_bits=bits)
    o = O.Index(p, ids, dim=dim, kind=KIND[kind], phi=32, bits=bits)
    if kind == "porth":
        check_porth_nodes(ix, o)
    else:
        check_spac_layout(ix, o)


@pytest.mark.parametrize("kind,dim,bits,n", [("spac_z", 2, 30, (1 << 20) + 17), ("spac_h", 2, 30, (1 << 20) + 3),
                                             ("porth", 2, 30, (1 << 20) + 9), ("spac_z", 3, 21, (1 << 20) + 1),
                                             ("spac_h", 3, 21, (1 << 20) + 11), ("porth", 3, 21, (1 << 20) + 5)])
def test_build_prefix_sort_runs(kind, dim, bits, n):
    # an encoding sort of at least 2^20 pairs whose keys take nearly n distinct
    # values in their top 48 bits (here: points in random order over the whole
    # domain) sorts those bits only, then puts each run of equal top bits in
    # (key, id) order.  Copies of existing points make runs of every kind:
    # 2..8 (fixed in registers), 20 and 300 (fixed in shared memory) and 5000
    # (fixed in global memory); the runs are few, so the prefix sort is taken.
    p = gen.uniform(n, dim, bits, 500 + n % 1000).astype(np.int32)
    rng = np.random.default_rng(n)
    src = rng.integers(0, n, 9000)
    pos = rng.permutation(n)[:len(src) + 5320]
    p[pos[:9000]] = p[src]                      # pairs and small runs
    for size, off in ((20, 9000), (300, 9020), (5000, 9320)):
        p[pos[off:off + size]] = p[src[size % 97]]  # piles of one point
    perm = np.argsort(gen.splitmix64(n, np.arange(n, dtype=np.uint64)), kind="stable").astype(np.uint64)
    with np.errstate(over="ignore"):
        ids = ((perm * np.uint64(2654435761) + np.uint64(7)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    dp, di = T(p), T(ids)
    psi.profile_enable(True)
    psi.profile_reset()
    ix = psi.Index(dp, di, kind=kind, leaf_size=32, coord_bits=bits)
    ix.sync()
    launched = psi.profile_dump()
    psi.profile_enable(False)
    assert "k_prefix_runs" in launched and "k_prefix_long" in launched  # the prefix sort was taken
    # input in random order: the gather reads points and ids from packed records
    assert any(name.startswith("k_pack_records") for name in launched)
    o = O.Index(p, ids, dim=dim, kind=KIND[kind], phi=32, bits=bits)
    if kind == "porth":
        check_porth_nodes(ix, o)
    else:
        check_spac_layout(ix, o)


@pytest.mark.parametrize("kind", ["spac_z", "spac_h"])
@pytest.mark.parametrize("dup", [False, True])
def test_spac_build_layout_3d_and_duplicates(kind, dup):
    p, ids = points(60000, 3, 21, 5, dup=dup)
    ix = psi.Index(T(p), T(ids), kind=kind, leaf_size=32, coord_bits=21)
    o = O.Index(p, ids, dim=3, kind=KIND[kind], phi=32, bits=21)
    check_spac_layout(ix, o)


def test_duplicate_pile_longer_than_a_tile():
    # 9000 copies of one point: equal keys must come out in id order
    p = np.zeros((9000, 2), np.int32) + 12345
    ids = np.random.default_rng(0).permutation(9000).astype(np.uint32) * 5
    ix = psi.Index(T(p), T(ids), kind="spac_z", leaf_size=32)
    check_spac_layout(ix, O.Index(p, ids, phi=32))


def test_build_rejects_out_of_range_coordinates():
    p = np.array([[0, 0], [1, (1 << 30) + 4]], np.int32)
    ix = psi.Index(T(p), T(np.arange(2, dtype=np.uint32)), kind="spac_z", coord_bits=30)
    with pytest.raises(psi.PsiError) as e:
        ix.sync()
    assert e.value.status == psi.ERR_RANGE


# ---------------------------------------------------------------- queries

def query_points(nq, dim, bits, seed, data):
    q = gen.uniform(nq, dim, bits, seed)
    if len(data):
        take = gen.sample_with_replacement(len(data), nq // 3, seed + 1)
        q[: nq // 3] = data[take]
    return q


@pytest.mark.parametrize("kind,dim", [("spac_h", 2), ("spac_z", 3)])
def test_knn_of_many_walk_ordered_queries(kind, dim):
    # 2^22 + 3 queries along random walks: the curve-order sort of the queries
    # packs its middle passes; every answer row must still belong to its query
    bits = 30 if dim == 2 else 21
    p, ids = points(200_000, dim, bits, 91, clustered=True)
    ix = psi.Index(T(p), T(ids), kind=kind, leaf_size=32, coord_bits=bits)
    o = O.Index(p, ids, dim=dim, kind=KIND[kind], phi=32, bits=bits)
    q = gen.varden((1 << 22) + 3, dim, bits, 92)
    gi, gd = ix.knn(T(q), 10)
    gi, gd = U32(gi), gd.cpu().numpy()
    rows = np.sort(gen.sample_with_replacement(len(q), 20_000, 93))
    oi, od = o.knn(q[rows], 10)
    assert (gi[rows] == oi).all() and (gd[rows] == od).all()


@pytest.mark.parametrize("kind,dim,bits", [("spac_z", 2, 30), ("spac_h", 2, 30), ("porth", 2, 30), ("spac_z", 3, 21),
                                           ("porth", 3, 21), ("spac_h", 3, 21)])
@pytest.mark.parametrize("k", [1, 10, 32, 33, 100, 128])
def test_knn_matches_oracle(kind, dim, bits, k):
    n = 30000
    p, ids = points(n, dim, bits, 21 + k, clustered=k % 2 == 0)
    ix = psi.Index(T(p), T(ids), kind=kind, leaf_size=32, coord_bits=bits)
    o = O.Index(p, ids, dim=dim, kind=KIND[kind], phi=32, bits=bits)
    q = query_points(5000, dim, bits, k, p)  # >= 4096: exercises the curve-sorted query order
    gi, gd = ix.knn(T(q), k)
    oi, od = o.knn(q, k)
    assert (U32(gi) == oi).all()
    assert (gd.cpu().numpy() == od).all()


@pytest.mark.parametrize("kind,dim,bits,n,phi,k,nq,dup", [("spac_h", 2, 30, 30000, 64, 10, 4097, False),
                                                         ("porth", 2, 30, 20000, 8, 5, 4099, True),
                                                         ("spac_z", 3, 21, 7, 32, 10, 4098, False),
                                                         ("spac_h", 2, 30, 50000, 32, 32, 4101, True),
                                                         ("spac_h", 3, 21, 40000, 16, 1, 4103, False)])
def test_knn_grouped_queries_ragged(kind, dim, bits, n, phi, k, nq, dup):
    # >= 4096 queries with k <= 32 run several curve-ordered queries per warp;
    # query counts not a multiple of the group size leave a short last group
    p, ids = points(n, dim, bits, 61 + nq, dup=dup, clustered=not dup)
    ix = psi.Index(T(p), T(ids), kind=kind, leaf_size=phi, coord_bits=bits)
    o = O.Index(p, ids, dim=dim, kind=KIND[kind], phi=phi, bits=bits)
    q = query_points(nq, dim, bits, 7 + k, p)
    gi, gd = ix.knn(T(q), k)
    oi, od = o.knn(q, k)
    assert (U32(gi) == oi).all()
    assert (gd.cpu().numpy() == od).all()
    si, sd, st = ix.knn_stats(T(q), k)
    assert torch.equal(si, gi) and torch.equal(sd, gd) and st["queries"] == nq


@pytest.mark.parametrize("n", [0, 1, 7, 40])
def test_knn_small_and_k_beyond_size(n):
    p, ids = points(n, 2, 30, 3)
    ix = psi.Index(T(p), T(ids), kind="spac_h", leaf_size=4, fanout=2)
    q = query_points(50, 2, 30, 5, p)
    gi, gd = ix.knn(T(q), 64)
    oi, od = O.knn_brute_raw(p.reshape(-1, 2), ids, q, 64)
    assert (U32(gi) == oi).all() and (gd.cpu().numpy() == od).all()


def test_knn_ties_by_id():
    # every point at the same distance from the query
    p = np.array([[10, 0], [0, 10], [20, 10], [10, 20]] * 50, np.int32)
    p[4:] += np.repeat(np.arange(1, 50), 4)[:, None].astype(np.int32) * 1000
    ids = np.random.default_rng(1).permutation(200).astype(np.uint32)
    ix = psi.Index(T(p), T(ids), kind="spac_z", leaf_size=2, fanout=2)
    gi, gd = ix.knn(T(np.array([[10, 10]], np.int32)), 4)
    want = sorted(ids[:4].tolist())
    assert U32(gi)[0].tolist() == want and gd.cpu().tolist()[0] == [100] * 4


@pytest.mark.parametrize("kind,dim,bits", [("spac_z", 2, 30), ("spac_h", 2, 30), ("porth", 2, 30), ("porth", 3, 21),
                                           ("spac_z", 3, 21), ("spac_h", 3, 21)])
def test_range_count_and_report_match_oracle(kind, dim, bits):
    n = 40000
    p, ids = points(n, dim, bits, 31, clustered=True)
    ix = psi.Index(T(p), T(ids), kind=kind, leaf_size=32, coord_bits=bits)
    o = O.Index(p, ids, dim=dim, kind=KIND[kind], phi=32, bits=bits)
    nq = 700
    centres = p[gen.sample_with_replacement(n, nq, 4)].astype(np.int64)
    half = np.int64(1) << np.int64(bits - 7)
    boxes = gen.centred_boxes(centres, int(half), bits)
    boxes[0, :dim], boxes[0, dim:] = 0, (1 << bits) - 1     # everything
    boxes[1, :dim], boxes[1, dim:] = p[5], p[5]             # a point
    boxes[2, :dim], boxes[2, dim:] = 9, 8                   # empty (lo > hi)
    gc = ix.range_count(T(boxes)).cpu().numpy()
    oc = o.range_count(boxes)
    assert (gc == oc).all()
    off, rid = ix.range_report(T(boxes), sort=True)
    ooff, orid = o.range_report(boxes)
    assert (off.cpu().numpy() == ooff).all()
    assert (U32(rid) == orid).all()
    # unsorted report: same sets
    off2, rid2 = ix.range_report(T(boxes), capacity=10)  # forces the capacity retry path
    r2 = U32(rid2)
    for t in range(0, nq, 37):
        a, b = ooff[t], ooff[t + 1]
        assert sorted(r2[a:b].tolist()) == orid[a:b].tolist()


# ---------------------------------------------------------------- updates

def spac_invariants(ix):
    gl = ix.leaves()
    gp = ix.points()
    leaf = gp["leaf"].cpu().numpy()
    keys, ids, pts = U64(gp["keys"]), U32(gp["ids"]), gp["pts"].cpu().numpy()
    cnt = gl["count"].cpu().numpy()
    assert (cnt > 0).all() and (cnt <= 2 * ix.leaf_size).all()
    assert np.bincount(leaf, minlength=len(cnt)).tolist() == cnt.tolist()
    lo, hi = gl["lo"].cpu().numpy(), gl["hi"].cpu().numpy()
    for d in range(ix.dim):
        mn = np.full(len(cnt), np.iinfo(np.int32).max)
        mx = np.full(len(cnt), np.iinfo(np.int32).min)
        np.minimum.at(mn, leaf, pts[:, d])
        np.maximum.at(mx, leaf, pts[:, d])
        assert (mn == lo[:, d]).all() and (mx == hi[:, d]).all()  # tight boxes
    # every point lies in its leaf's (key, id) range [sep_j, sep_{j+1})
    sk, si = U64(gl["sep_key"]), U32(gl["sep_id"])
    pair = keys.astype(object) * (1 << 32) + ids.astype(object)
    sep = sk.astype(object) * (1 << 32) + si.astype(object)
    nxt = np.append(sep[1:], np.array([1 << 100], dtype=object))
    assert all(sep[1:] > sep[:-1])
    assert all((pair < nxt[leaf]) & ((pair >= sep[leaf]) | (leaf == 0)))
    # the leaf wrap (Sec 4.2): every leaf but the index's last holds at least phi / 2 points
    assert (cnt[:-1] >= max(1, ix.leaf_size // 2)).all()


@pytest.mark.parametrize("kind,dim,bits,phi", [("spac_z", 2, 30, 32), ("spac_h", 2, 30, 32), ("porth", 2, 30, 32),
                                               ("spac_h", 3, 21, 32), ("porth", 3, 21, 32),
                                               ("spac_h", 2, 30, 64), ("spac_z", 3, 21, 64), ("spac_z", 2, 30, 64),
                                               ("spac_h", 3, 21, 64), ("porth", 3, 21, 64)])
def test_updates_match_oracle(kind, dim, bits, phi):
    # phi = 64: leaf blocks of 128 slots, so the update kernels run their
    # four-rows-per-lane instances
    n = 50000
    p, ids = points(n, dim, bits, 41, clustered=True)
    ix = psi.Index(T(p), T(ids), kind=kind, leaf_size=phi, coord_bits=bits)
    o = O.Index(p, ids, dim=dim, kind=KIND[kind], phi=phi, bits=bits)
    live_p, live_i = p, ids
    rng_seed = 5
    for step, (m_ins, m_del, ood) in enumerate([(5000, 3000, False), (20000, 1000, True), (100, 30000, False),
                                                (60000, 0, True), (0, 50000, False)]):
        newp = gen.varden(m_ins, dim, bits, 1000 + step, x_range=(1 << (bits - 1), 1 << bits) if ood else None)
        newi = (np.arange(m_ins, dtype=np.uint32) + 10_000_000 * (step + 1)).astype(np.uint32)
        ix.insert(T(newp), T(newi))
        o.insert(newp, newi)
        live_p = np.concatenate([live_p, newp])
        live_i = np.concatenate([live_i, newi])
        sel = gen.sample_without_replacement(len(live_i), min(m_del, len(live_i)), rng_seed + step)
        dp = np.concatenate([live_p[sel], [[3, 4, 5][:dim]]]).astype(np.int32)   # plus one absent point
        di = np.concatenate([live_i[sel], [live_i[0]]]).astype(np.uint32)
        nd = torch.zeros(1, dtype=torch.int64, device=DEV)
        ix.delete(T(dp), T(di), nd)
        got_del = int(nd.item())
        want_del = o.delete(dp, di)
        assert got_del == want_del == len(sel)
        keep = np.ones(len(live_i), bool)
        keep[sel] = False
        live_p, live_i = live_p[keep], live_i[keep]
        ix.sync()
        assert len(ix) == len(o) == len(live_i)
        # point sets
        gp = ix.points()
        ok, oi, op = o.points()
        gi = U32(gp["ids"])
        order = np.argsort(gi)
        oorder = np.argsort(oi)
        assert (gi[order] == oi[oorder]).all()
        assert (gp["pts"].cpu().numpy()[order] == op[oorder]).all()
        if kind != "porth" and len(live_i):
            spac_invariants(ix)
        # queries
        q = query_points(3000, dim, bits, 7 + step, live_p)
        gi, gd = ix.knn(T(q), 10)
        oi2, od2 = o.knn(q, 10)
        assert (U32(gi) == oi2).all() and (gd.cpu().numpy() == od2).all()
        boxes = gen.square_boxes(300, dim, bits, 1 << (bits - 7), 9 + step)
        assert (ix.range_count(T(boxes)).cpu().numpy() == o.range_count(boxes)).all()
        # range lists (and counts) of boxes centred on live points, over leaves of up
        # to 2 phi points (more than one 32-lane round)
        if len(live_p):
            rb = gen.centred_boxes(live_p[gen.sample_with_replacement(len(live_p), 60, 29 + step)], 1 << (bits - 6),
                                   bits)
            assert (ix.range_count(T(rb)).cpu().numpy() == o.range_count(rb)).all()
            off, rid = ix.range_report(T(rb), sort=True)
            ooff, orid = o.range_report(rb)
            assert (off.cpu().numpy() == ooff).all() and (U32(rid) == orid).all()
        if kind == "porth":
            check_porth_nodes(ix, o)


@pytest.mark.parametrize("kind,dim,bits,phi", [("spac_h", 2, 30, 8), ("spac_z", 3, 21, 32), ("spac_h", 2, 30, 2),
                                               ("spac_z", 2, 30, 64), ("spac_h", 3, 21, 4)])
def test_delete_restores_the_leaf_wrap(kind, dim, bits, phi):
    # deletes that leave long runs of underfull and empty leaves, in the middle
    # and at the end of the key order, then a delete of almost everything
    n = 200_000
    p, ids = points(n, dim, bits, 71 + phi, clustered=True)
    ix = psi.Index(T(p), T(ids), kind=kind, leaf_size=phi, coord_bits=bits)
    o = O.Index(p, ids, dim=dim, kind=KIND[kind], phi=phi, bits=bits)
    order = np.lexsort((ids, O.keys(p, dim, KIND[kind], bits)))  # (key, id) order
    live = np.ones(n, bool)
    rng = np.random.default_rng(phi)
    steps = [order[20_000:120_000][rng.random(100_000) < 0.93],   # a long run of underfull leaves
             order[130_000:131_000],                               # a run of emptied leaves
             order[190_000:][rng.random(10_000) < 0.99],           # the tail of the key order
             order[rng.random(n) < 0.999]]                         # almost everything
    for sel in steps:
        sel = sel[live[sel]]
        nd = torch.zeros(1, dtype=torch.int64, device=DEV)
        ix.delete(T(p[sel]), T(ids[sel]), nd)
        assert int(nd.item()) == o.delete(p[sel], ids[sel]) == len(sel)
        live[sel] = False
        ix.sync()
        assert len(ix) == len(o) == int(live.sum())
        gp = ix.points()
        gi = np.sort(U32(gp["ids"]))
        assert (gi == np.sort(ids[live])).all()
        if len(ix):
            spac_invariants(ix)
        q = query_points(2000, dim, bits, 5 + phi, p[live] if live.any() else p)
        gi, gd = ix.knn(T(q), 10)
        oi, od = o.knn(q, 10)
        assert (U32(gi) == oi).all() and (gd.cpu().numpy() == od).all()
    # inserts after the re-wraps land in the new leaves
    newp = gen.varden(30_000, dim, bits, 99)
    newi = (np.arange(30_000) + 50_000_000).astype(np.uint32)
    ix.insert(T(newp), T(newi))
    o.insert(newp, newi)
    ix.sync()
    spac_invariants(ix)
    q = query_points(2000, dim, bits, 6, newp)
    gi, gd = ix.knn(T(q), 10)
    oi, od = o.knn(q, 10)
    assert (U32(gi) == oi).all() and (gd.cpu().numpy() == od).all()


@pytest.mark.parametrize("kind", ["spac_z", "spac_h"])
def test_inserts_below_the_first_key_keep_separators_increasing(kind):
    # leaf 0 is open below: points under its separator are appended to it, and
    # when it overflows its re-wrapped parts must keep the separators
    # increasing, or later batches would be routed to the wrong leaves
    bits = 30
    p, ids = points(5000, 2, bits, 81)
    p = p | (1 << 20)  # every base point away from the curve's start at (0, 0)
    ix = psi.Index(T(p), T(ids), kind=kind, leaf_size=8, coord_bits=bits)
    o = O.Index(p, ids, kind=KIND[kind], phi=8, bits=bits)
    for step in range(3):
        lowp = (gen.uniform(40, 2, bits, 7 + step) >> 12).astype(np.int32)  # keys below every base key
        lowi = (np.arange(40) + 1_000_000 * (step + 1)).astype(np.uint32)
        ix.insert(T(lowp), T(lowi))
        o.insert(lowp, lowi)
        ix.sync()
        spac_invariants(ix)
    # every low point can be deleted again (it is routed to the leaf holding it)
    lo_all = np.concatenate([(gen.uniform(40, 2, bits, 7 + st) >> 12).astype(np.int32) for st in range(3)])
    lo_ids = np.concatenate([(np.arange(40) + 1_000_000 * (st + 1)).astype(np.uint32) for st in range(3)])
    nd = torch.zeros(1, dtype=torch.int64, device=DEV)
    ix.delete(T(lo_all), T(lo_ids), nd)
    assert int(nd.item()) == o.delete(lo_all, lo_ids) == 120
    ix.sync()
    spac_invariants(ix)
    gi = np.sort(U32(ix.points()["ids"]))
    assert (gi == np.sort(ids)).all()


def test_insert_into_empty_and_delete_everything():
    ix = psi.Index(T(np.zeros((0, 2), np.int32)), T(np.zeros(0, np.uint32)), kind="spac_h")
    p, ids = points(3000, 2, 30, 8)
    ix.insert(T(p), T(ids))
    o = O.Index(p, ids, kind=O.SPAC_H)
    check_spac_layout(ix, o)
    ix.delete(T(p), T(ids))
    ix.sync()
    assert len(ix) == 0 and ix.num_leaves == 0
    gi, gd = ix.knn(T(p[:5]), 3)
    assert (U32(gi) == 0xFFFFFFFF).all()


# ---------------------------------------------------------------- P-Orth

def check_porth_nodes(ix, o):
    want = o.porth()
    nd = ix.nodes()
    D, bits = ix.dim, ix.coord_bits
    depth = nd["depth"].cpu().numpy()
    prefix = U64(nd["prefix"])
    start = np.array([int(pr) << (D * (bits - int(dd))) for pr, dd in zip(prefix, depth)], dtype=object)
    order = sorted(range(len(depth)), key=lambda i: (start[i], depth[i]))
    assert len(order) == len(want["depth"])
    o_ = np.array(order, dtype=np.int64)
    assert (depth[o_] == want["depth"]).all()
    assert (prefix[o_] == want["prefix"]).all()
    assert (nd["count"].cpu().numpy()[o_] == want["count"]).all()
    assert (nd["lo"].cpu().numpy()[o_] == want["lo"]).all()
    assert (nd["hi"].cpu().numpy()[o_] == want["hi"]).all()
    assert (nd["is_leaf"].cpu().numpy()[o_] == want["is_leaf"]).all()


@pytest.mark.parametrize("dim,bits,phi,clustered,dup", [(2, 30, 32, False, False), (2, 30, 32, True, False),
                                                        (2, 30, 8, True, True), (3, 21, 32, True, False),
                                                        (3, 21, 16, False, True), (2, 10, 4, False, False)])
def test_porth_build_matches_oracle(dim, bits, phi, clustered, dup):
    p, ids = points(40000, dim, bits, 51 + phi, dup=dup, clustered=clustered)
    ix = psi.Index(T(p), T(ids), kind="porth", leaf_size=phi, coord_bits=bits)
    o = O.Index(p, ids, dim=dim, kind=O.PORTH, phi=phi, bits=bits)
    check_porth_nodes(ix, o)


@pytest.mark.parametrize("dim,bits,phi", [(2, 30, 8), (3, 21, 32), (2, 30, 32)])
def test_porth_local_updates_match_a_fresh_build(dim, bits, phi):
    # many small batches: each rebuilds only the leaves within phi + 1 points
    # of a changed point; after every batch the node list must equal the
    # canonical tree of the new point set
    n = 40000
    p, ids = points(n, dim, bits, 300 + phi, clustered=True)
    ix = psi.Index(T(p), T(ids), kind="porth", leaf_size=phi, coord_bits=bits)
    o = O.Index(p, ids, dim=dim, kind=O.PORTH, phi=phi, bits=bits)
    live_p, live_i = p.copy(), ids.copy()
    rng = np.random.default_rng(phi + dim)
    next_id = 10_000_000
    for step in range(16):
        kind = step % 4
        if kind in (0, 2):   # insert: new points, copies of existing points (duplicate piles), far points
            mi = int(rng.integers(1, 300))
            newp = gen.varden(mi, dim, bits, 400 + step)
            cp = live_p[rng.integers(0, len(live_p), mi // 3 + 1)]
            far = gen.uniform(3, dim, bits, 500 + step)
            newp = np.concatenate([newp, cp, cp[:2], far]).astype(np.int32)
            newi = (np.arange(len(newp)) + next_id).astype(np.uint32)
            next_id += len(newp)
            ix.insert(T(newp), T(newi))
            o.insert(newp, newi)
            live_p = np.concatenate([live_p, newp])
            live_i = np.concatenate([live_i, newi])
        else:                # delete: live points (a whole neighbourhood when kind == 3) and absent ones
            md = int(rng.integers(1, 300))
            if kind == 3:
                c = rng.integers(0, len(live_p))
                d2 = ((live_p.astype(np.int64) - live_p[c].astype(np.int64)) ** 2).sum(1)
                sel = np.argsort(d2, kind="stable")[:md]
            else:
                sel = rng.choice(len(live_p), md, replace=False)
            dp = np.concatenate([live_p[sel], gen.uniform(2, dim, bits, 600 + step)]).astype(np.int32)
            di = np.concatenate([live_i[sel], [0xFFFFFFF0, 0xFFFFFFF1]]).astype(np.uint32)
            nd = torch.zeros(1, dtype=torch.int64, device=DEV)
            ix.delete(T(dp), T(di), nd)
            assert int(nd.item()) == o.delete(dp, di) == len(sel)
            keep = np.ones(len(live_i), bool)
            keep[sel] = False
            live_p, live_i = live_p[keep], live_i[keep]
        ix.sync()
        assert len(ix) == len(o) == len(live_i)
        check_porth_nodes(ix, o)
    q = query_points(3000, dim, bits, 9, live_p)
    for k in (10, 100):
        gi, gd = ix.knn(T(q), k)
        oi, od = o.knn(q, k)
        assert (U32(gi) == oi).all() and (gd.cpu().numpy() == od).all()
    # delete everything, then insert into the empty tree
    nd = torch.zeros(1, dtype=torch.int64, device=DEV)
    ix.delete(T(live_p), T(live_i), nd)
    ix.sync()
    assert int(nd.item()) == len(live_i) and len(ix) == 0 and ix.num_nodes == 0
    ix.insert(T(p[:5000]), T(ids[:5000]))
    ix.sync()
    check_porth_nodes(ix, O.Index(p[:5000], ids[:5000], dim=dim, kind=O.PORTH, phi=phi, bits=bits))


def test_porth_tiny():
    for n in (0, 1, 2, 33):
        p, ids = points(n, 2, 30, 3 + n)
        ix = psi.Index(T(p), T(ids), kind="porth", leaf_size=32)
        o = O.Index(p, ids, kind=O.PORTH, phi=32)
        if n:
            check_porth_nodes(ix, o)
        else:
            assert ix.num_nodes == 0
