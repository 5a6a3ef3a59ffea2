"""Pins of the oracle's P-Orth tree (Algorithm 1) against an independent
construction by cell arithmetic and a hand-checked example."""
import numpy as np
import pytest

from oracle import oracle as O


def porth_by_cells(pts, phi, bits):
    """Node (depth l, cell c) exists iff l == 0, or its parent cell at depth l-1
    exists, holds more than phi points and is not a single grid cell.  Cell of p
    at depth l is p >> (bits - l) per coordinate.  Returns nodes sorted in
    preorder with (depth, prefix, count, lo, hi, is_leaf)."""
    n, D = pts.shape
    if n == 0:
        return []
    P = pts.astype(np.int64)
    nodes = []
    alive = np.ones(n, bool)      # points whose depth-l cell is a node
    for l in range(bits + 1):
        if not alive.any():
            break
        cells = P[alive] >> (bits - l)
        uniq, inv, cnt = np.unique(cells, axis=0, return_inverse=True, return_counts=True)
        inv = inv.reshape(-1)
        split = np.zeros(len(uniq), bool)
        sub = P[alive]
        for u in range(len(uniq)):
            mem = sub[inv == u]
            # prefix: child numbers of the levels above, most significant first
            prefix = 0
            for j in range(l):
                bitpos = bits - 1 - j
                child = sum((((int(uniq[u][d]) << (bits - l)) >> bitpos) & 1) << d for d in range(D))
                prefix = (prefix << D) | child
            leaf = cnt[u] <= phi or l == bits
            split[u] = not leaf
            nodes.append((l, prefix, int(cnt[u]), tuple(mem.min(0)), tuple(mem.max(0)), int(leaf)))
        idx = np.flatnonzero(alive)
        alive[idx[~split[inv]]] = False
    # preorder: by the first key of the cell's range, parents before children
    nodes.sort(key=lambda t: (t[1] << (D * (bits - t[0])), t[0]))
    return nodes


def oracle_nodes(ix):
    t = ix.porth()
    return [(int(t["depth"][i]), int(t["prefix"][i]), int(t["count"][i]), tuple(t["lo"][i]), tuple(t["hi"][i]),
             int(t["is_leaf"][i])) for i in range(len(t["depth"]))]


def test_porth_hand_example():
    # domain 4x4 (b = 2), phi = 1: root splits; quadrant 0 holds two points and splits again
    pts = np.array([[0, 0], [3, 3], [1, 1]], np.int32)
    ix = O.Index(pts, np.arange(3, dtype=np.uint32), kind=O.PORTH, phi=1, bits=2)
    assert oracle_nodes(ix) == [
        (0, 0, 3, (0, 0), (3, 3), 0),
        (1, 0, 2, (0, 0), (1, 1), 0),
        (2, 0, 1, (0, 0), (0, 0), 1),
        (2, 3, 1, (1, 1), (1, 1), 1),
        (1, 3, 1, (3, 3), (3, 3), 1),
    ]


@pytest.mark.parametrize("dim,bits,phi,hi", [(2, 10, 4, 1 << 10), (2, 10, 4, 40), (3, 7, 3, 1 << 7), (2, 30, 8, 1 << 30)])
def test_porth_matches_cell_definition(dim, bits, phi, hi):
    rng = np.random.default_rng(bits + dim)
    pts = rng.integers(0, hi, size=(1500, dim)).astype(np.int32)
    pts[:50] = pts[0]  # a pile of duplicates forces the depth-b rule
    ix = O.Index(pts, np.arange(len(pts), dtype=np.uint32), dim=dim, kind=O.PORTH, phi=phi, bits=bits)
    got = oracle_nodes(ix)
    assert got == porth_by_cells(pts, phi, bits)
    # structure: counts of children add up; leaves hold <= phi unless at depth b
    for d, p, c, lo, hi_, leaf in got:
        if leaf:
            assert c <= phi or d == bits
    assert got[0][2] == len(pts)


def test_porth_history_independent_after_updates():
    rng = np.random.default_rng(5)
    a = rng.integers(0, 1 << 12, size=(800, 2)).astype(np.int32)
    b = rng.integers(0, 1 << 12, size=(400, 2)).astype(np.int32)
    ix = O.Index(a, np.arange(800, dtype=np.uint32), kind=O.PORTH, phi=6, bits=12)
    ix.insert(b, np.arange(800, 1200, dtype=np.uint32))
    ix.delete(a[:300], np.arange(300, dtype=np.uint32))
    live = np.concatenate([a[300:], b])
    assert oracle_nodes(ix) == porth_by_cells(live, 6, 12)
