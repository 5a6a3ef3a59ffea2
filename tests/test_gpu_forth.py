"""The float P-Orth (SFC-free construction, Sec 3 / Algorithm 1) against the
float oracle: node arrays in breadth-first order, leaf contents, k-NN (ids and
double squared distances, bit-exact) and range counts, for D = 2..5."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2601_05347_gb300 import psi


def T(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to("cuda")


def points(n, dim, seed, lo=0.0, hi=1.0, clustered=False, dup=0):
    rng = np.random.default_rng(seed)
    if clustered:
        c = rng.random((20, dim)) * (hi - lo) + lo
        p = c[rng.integers(0, 20, n)] + rng.normal(0, 0.01 * (hi - lo), (n, dim))
    else:
        p = rng.random((n, dim)) * (hi - lo) + lo
    p = np.clip(p, lo, np.nextafter(np.float32(hi), np.float32(lo))).astype(np.float32)
    if dup:
        p[:dup] = p[0]
    ids = rng.permutation(n).astype(np.uint32) * 3 + 1
    return p, ids


def check_tree(f, o):
    g = {k: v.cpu().numpy() for k, v in f.nodes().items()}
    on = o.nodes()
    assert len(g["depth"]) == len(on["depth"])
    assert (g["depth"] == on["depth"]).all()
    assert (g["count"] == on["count"]).all()
    assert (g["kids"] == on["kids"]).all()
    assert ((g["kids"] == 0) == (on["is_leaf"] == 1)).all()
    assert (g["lo"].view(np.int32) == on["lo"].view(np.int32)).all()
    assert (g["hi"].view(np.int32) == on["hi"].view(np.int32)).all()
    gid = g["ids"].view(np.uint32)
    for u in np.flatnonzero(on["is_leaf"]):
        r, c, a = int(g["ref"][u]), int(g["count"][u]), int(on["leaf_first"][u])
        assert (np.sort(gid[r:r + c]) == on["leaf_ids"][a:a + c]).all(), u


@pytest.mark.parametrize("dim,phi,clustered", [(2, 4, False), (2, 32, True), (3, 16, False), (3, 32, True),
                                                (4, 8, False), (5, 32, False), (5, 6, True)])
def test_build_matches_oracle(dim, phi, clustered):
    p, ids = points(20000, dim, 7 * dim + phi, clustered=clustered)
    f = psi.FOrth(T(p), T(ids), [0] * dim, [1] * dim, leaf_size=phi)
    o = O.FOrth(p, ids, [0] * dim, [1] * dim, phi=phi)
    check_tree(f, o)
    f.close()


def test_duplicates_and_a_negative_region():
    p, ids = points(5000, 3, 3, lo=-100.0, hi=100.0, dup=300)
    f = psi.FOrth(T(p), T(ids), [-100] * 3, [100] * 3, leaf_size=8)
    o = O.FOrth(p, ids, [-100] * 3, [100] * 3, phi=8)
    check_tree(f, o)
    g = f.nodes()
    assert int(g["count"][g["kids"] == 0].max()) >= 300  # the pile is one leaf (precision exhausted)


@pytest.mark.parametrize("dim", [2, 3, 4, 5])
@pytest.mark.parametrize("k", [1, 10, 33, 100])
def test_knn_matches_oracle(dim, k):
    p, ids = points(15000, dim, 11 * dim + k, clustered=k % 2 == 0)
    rng = np.random.default_rng(k)
    q = rng.random((5000, dim)).astype(np.float32)  # >= 4096: the curve-ordered query path
    q[:2000] = p[rng.integers(0, len(p), 2000)]
    f = psi.FOrth(T(p), T(ids), [0] * dim, [1] * dim, leaf_size=16)
    gi, gd = f.knn(T(q), k)
    f.sync()
    oi, od = O.fknn_brute(p, ids, q, k)
    assert (gi.cpu().numpy().view(np.uint32) == oi).all()
    assert (gd.cpu().numpy().view(np.int64) == od.view(np.int64)).all()


@pytest.mark.parametrize("dim", [2, 3, 5])
def test_range_count_matches_oracle(dim):
    p, ids = points(30000, dim, 5 + dim, clustered=True)
    rng = np.random.default_rng(dim)
    c = p[rng.integers(0, len(p), 800)]
    h = rng.random((800, 1)).astype(np.float32) * 0.05
    boxes = np.concatenate([c - h, c + h], axis=1).astype(np.float32)
    boxes[:5, :dim] = 2.0  # empty boxes (lo > hi)
    f = psi.FOrth(T(p), T(ids), [0] * dim, [1] * dim, leaf_size=32)
    got = f.range_count(T(boxes)).cpu().numpy()
    assert (got == O.frange_count_brute(p, boxes)).all()


def test_updates_equal_a_fresh_build():
    dim = 3
    p, ids = points(12000, dim, 21, clustered=True)
    q, qids = points(4000, dim, 22)
    qids = qids + 1_000_000
    f = psi.FOrth(T(p), T(ids), [0] * dim, [1] * dim, leaf_size=8)
    f.insert(T(q), T(qids))
    nd = torch.zeros(1, dtype=torch.int64, device="cuda")
    dele = np.concatenate([p[::3], [[0.5, 0.5, 0.5]]]).astype(np.float32)  # plus one absent point
    deli = np.concatenate([ids[::3], [ids[1]]]).astype(np.uint32)
    f.delete(T(dele), T(deli), nd)
    assert int(nd.item()) == len(p[::3])
    keep = np.ones(len(p), bool)
    keep[::3] = False
    live_p = np.concatenate([p[keep], q])
    live_i = np.concatenate([ids[keep], qids])
    assert len(f) == len(live_p)
    check_tree(f, O.FOrth(live_p, live_i, [0] * dim, [1] * dim, phi=8))
    gi, gd = f.knn(T(q[:500]), 10)
    oi, od = O.fknn_brute(live_p, live_i, q[:500], 10)
    assert (gi.cpu().numpy().view(np.uint32) == oi).all() and (gd.cpu().numpy() == od).all()


def test_empty_and_out_of_region():
    f = psi.FOrth(T(np.zeros((0, 2), np.float32)), T(np.zeros(0, np.uint32)), [0, 0], [1, 1])
    gi, gd = f.knn(T(np.array([[0.5, 0.5]], np.float32)), 3)
    assert gi.cpu().numpy().view(np.uint32).tolist() == [[0xFFFFFFFF] * 3]
    assert np.isinf(gd.cpu().numpy()).all()
    f.insert(T(np.array([[0.25, 0.75]], np.float32)), T(np.array([9], np.uint32)))
    gi, gd = f.knn(T(np.array([[0.5, 0.5]], np.float32)), 2)
    assert gi.cpu().numpy().view(np.uint32).tolist()[0][0] == 9 and gd.cpu().numpy()[0][0] == 0.125
    with pytest.raises(psi.PsiError):
        psi.FOrth(T(np.array([[1.0, 0.5]], np.float32)), T(np.array([0], np.uint32)), [0, 0], [1, 1])
