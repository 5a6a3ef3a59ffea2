"""Pins of the float P-Orth oracle (SFC-free construction, Sec 3.1 / Algorithm 1).

The oracle builds the tree as a breadth-first recursion over regions.  It is
checked against: the integer P-Orth oracle (built from Morton cells) on
integer-valued points, a vectorised restatement of the node definition for
higher dimensions, brute-force integer k-NN and range counts, and a hand example."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2601_05347_gb300 import gen


def node_rows(depth, count, lo, hi, is_leaf):
    rows = [(int(d), tuple(float(x) for x in l), tuple(float(x) for x in h), int(c), int(f))
            for d, c, l, h, f in zip(depth, count, lo, hi, is_leaf)]
    return sorted(rows)


@pytest.mark.parametrize("dim,bits,phi", [(2, 10, 4), (2, 12, 32), (3, 7, 8), (3, 9, 32)])
@pytest.mark.parametrize("clustered", [False, True])
def test_integer_points_give_the_integer_porth(dim, bits, phi, clustered):
    n = 3000
    p = gen.varden(n, dim, bits, 5, step=4) if clustered else gen.uniform(n, dim, bits, 6)
    ids = np.arange(n, dtype=np.uint32)
    f = O.FOrth(p.astype(np.float32), ids, [0] * dim, [1 << bits] * dim, phi=phi, max_depth=bits)
    fn = f.nodes()
    o = O.Index(p, ids, dim=dim, kind=O.PORTH, phi=phi, bits=bits)
    on = o.porth()
    assert len(fn["depth"]) == len(on["depth"])
    assert node_rows(fn["depth"], fn["count"], fn["lo"], fn["hi"], fn["is_leaf"]) == node_rows(
        on["depth"], on["count"], on["lo"].astype(np.float32), on["hi"].astype(np.float32), on["is_leaf"])


def definition_nodes(p, lo, hi, phi, max_depth):
    """Nodes by definition: the cells of each depth (computed per point with the
    float midpoint rule) that hold a point and whose parent cell holds more than
    phi points and can still be split."""
    n, D = p.shape
    clo = np.tile(np.asarray(lo, np.float32), (n, 1))
    chi = np.tile(np.asarray(hi, np.float32), (n, 1))
    path = [tuple()] * n
    rows = []
    alive = np.ones(n, bool)  # the point's cell at this depth is a node
    for depth in range(max_depth + 1):
        keys = {}
        for i in np.flatnonzero(alive):
            keys.setdefault(path[i], []).append(i)
        mid = (clo + np.float32(0.5) * (chi - clo)).astype(np.float32)
        splittable = np.all((clo < mid) & (mid < chi), axis=1)
        nxt = np.zeros(n, bool)
        for key, members in keys.items():
            members = np.asarray(members)
            leaf = len(members) <= phi or depth == max_depth or not splittable[members[0]]
            rows.append((depth, tuple(float(x) for x in p[members].min(0)), tuple(float(x) for x in p[members].max(0)),
                         len(members), int(leaf)))
            if not leaf:
                nxt[members] = True
        if not nxt.any():
            break
        up = p >= mid
        clo = np.where(up, mid, clo).astype(np.float32)
        chi = np.where(up, chi, mid).astype(np.float32)
        path = [path[i] + (int(np.dot(up[i], 1 << np.arange(D))),) if nxt[i] else path[i] for i in range(n)]
        alive = nxt
    return sorted(rows)


@pytest.mark.parametrize("dim", [2, 4, 5])
def test_node_definition_in_higher_dimensions(dim):
    rng = np.random.default_rng(dim)
    n = 1500
    p = np.concatenate([rng.random((n // 2, dim)), 0.3 + 0.01 * rng.random((n - n // 2, dim))]).astype(np.float32)
    lo, hi = [0.0] * dim, [1.0] * dim
    f = O.FOrth(p, np.arange(n), lo, hi, phi=6, max_depth=30)
    fn = f.nodes()
    got = node_rows(fn["depth"], fn["count"], fn["lo"], fn["hi"], fn["is_leaf"])
    assert got == definition_nodes(p, lo, hi, 6, 30)
    # breadth-first layout: depths non-decreasing, children consecutive
    assert (np.diff(fn["depth"]) >= 0).all()
    internal = np.flatnonzero(fn["is_leaf"] == 0)
    assert fn["count"][0] == n and fn["kids"][internal].sum() == len(fn["depth"]) - 1
    # the leaves' ids partition the point set
    ids = np.sort(fn["leaf_ids"][:n])
    assert (ids == np.arange(n)).all()


def test_precision_exhaustion_makes_a_leaf():
    # 100 copies of one point (and its float neighbour): no split can separate them
    x = np.float32(0.3)
    p = np.array([[x, x]] * 50 + [[np.nextafter(x, np.float32(1)), x]] * 50, np.float32)
    f = O.FOrth(p, np.arange(100), [0, 0], [1, 1], phi=4, max_depth=60)
    fn = f.nodes()
    leaves = np.flatnonzero(fn["is_leaf"])
    assert sorted(fn["count"][leaves].tolist()) == [50, 50]
    assert fn["depth"].max() < 60  # stopped by exhausted precision, not by the depth cap


def test_hand_example():
    # H = [0, 8)^2, phi = 2: five points; the root splits at 4, the lower-left
    # quadrant (3 points) splits again at 2
    p = np.array([[1, 1], [1.5, 3], [3, 3], [6, 1], [7, 7]], np.float32)
    f = O.FOrth(p, np.arange(5), [0, 0], [8, 8], phi=2)
    fn = f.nodes()
    assert fn["depth"].tolist() == [0, 1, 1, 1, 2, 2, 2]
    assert fn["count"].tolist() == [5, 3, 1, 1, 1, 1, 1]
    assert fn["is_leaf"].tolist() == [0, 0, 1, 1, 1, 1, 1]
    # children of the lower-left quadrant: cell (0,0) holds (1,1), cell (0,1) holds (1.5,3), cell (1,1) holds (3,3)
    assert fn["lo"][4:].tolist() == [[1, 1], [1.5, 3], [3, 3]]


@pytest.mark.parametrize("dim", [2, 3])
def test_float_knn_and_counts_equal_integer_brute_force(dim):
    bits = 18  # squared distances stay exact in double
    n = 2000
    p = gen.uniform(n, dim, bits, 9)
    ids = (np.arange(n, dtype=np.uint32) * 7919) % 100003
    q = gen.uniform(300, dim, bits, 10)
    q[:50] = p[:50]
    fi, fd = O.fknn_brute(p.astype(np.float32), ids, q.astype(np.float32), 12)
    ii, idd = O.knn_brute_raw(p, ids, q, 12)
    assert (fi == ii).all() and (fd == idd.astype(np.float64)).all()
    boxes = gen.square_boxes(200, dim, bits, 1 << 14, 11)
    assert (O.frange_count_brute(p.astype(np.float32), boxes.astype(np.float32))
            == O.range_count_brute_raw(p, boxes)).all()


def test_knn_pads_beyond_size():
    p = np.array([[0.5, 0.5], [0.25, 0.75]], np.float32)
    i, d = O.fknn_brute(p, np.array([7, 3], np.uint32), np.array([[0.5, 0.5]], np.float32), 4)
    assert i[0].tolist() == [7, 3, 0xFFFFFFFF, 0xFFFFFFFF]
    assert d[0][0] == 0.0 and d[0][1] == 0.125 and np.isinf(d[0][2:]).all()


def test_points_outside_the_region_are_rejected():
    with pytest.raises(ValueError):
        O.FOrth(np.array([[1.0, 0.5]], np.float32), [0], [0, 0], [1, 1])
