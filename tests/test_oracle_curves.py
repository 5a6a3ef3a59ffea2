"""Pins of the oracle's space-filling curves against facts fixed by the curves'
definitions (Sec 2.2), not by retyping the oracle's formulas."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O


def z_order_cells(dim, bits):
    """Cells of [0,2^bits)^dim in Z-order, by recursive subdivision: a square is
    cut at its midpoint and the 2^dim sub-squares are visited in the order of
    their child number sum_d (upper half in d) << d."""
    out = []

    def rec(corner, side):
        if side == 1:
            out.append(tuple(corner))
            return
        h = side // 2
        for c in range(1 << dim):
            rec([corner[d] + (h if (c >> d) & 1 else 0) for d in range(dim)], h)

    rec([0] * dim, 1 << bits)
    return out


@pytest.mark.parametrize("dim,bits", [(2, 1), (2, 4), (3, 1), (3, 3)])
def test_morton_is_recursive_z_order(dim, bits):
    for rank, cell in enumerate(z_order_cells(dim, bits)):
        assert O.morton(cell, dim, bits) == rank


def test_morton_extremes():
    assert O.morton([1, 0], 2, 30) == 1
    assert O.morton([0, 1], 2, 30) == 2
    assert O.morton([(1 << 30) - 1] * 2, 2, 30) == (1 << 60) - 1
    assert O.morton([(1 << 21) - 1] * 3, 3, 21) == (1 << 63) - 1
    assert O.morton([0, 0, 1], 3, 21) == 4
    # the top bits of a coordinate land at the top of the key
    assert O.morton([1 << 29, 0], 2, 30) == 1 << 58
    assert O.morton([0, 1 << 29], 2, 30) == 1 << 59


def hilbert_inverse(bits):
    cells = [None] * (1 << (2 * bits))
    for x in range(1 << bits):
        for y in range(1 << bits):
            d = O.hilbert2(x, y, bits)
            assert 0 <= d < len(cells)
            assert cells[d] is None, "not a bijection"
            cells[d] = (x, y)
    return cells


def test_hilbert_order_one():
    # Hilbert's first-order curve visits the four cells in a U: up, right, down.
    assert hilbert_inverse(1) == [(0, 0), (0, 1), (1, 1), (1, 0)]


@pytest.mark.parametrize("bits", [2, 3, 4, 5, 6])
def test_hilbert_bijection_adjacency_endpoints_nesting(bits):
    cells = hilbert_inverse(bits)
    side = 1 << bits
    assert cells[0] == (0, 0)
    assert cells[-1] == (side - 1, 0)
    # consecutive indices are grid neighbours (Sec 5.1.3: adjacent codes are always geometrically close)
    for a, b in zip(cells, cells[1:]):
        assert abs(a[0] - b[0]) + abs(a[1] - b[1]) == 1
    # every aligned run of 4^j indices fills an aligned 2^j x 2^j square
    for j in range(1, bits):
        blk = 1 << (2 * j)
        for t in range(0, len(cells), blk):
            xs = {c[0] >> j for c in cells[t:t + blk]}
            ys = {c[1] >> j for c in cells[t:t + blk]}
            assert len(xs) == 1 and len(ys) == 1


def test_hilbert_quadrant_orientation():
    # the first quarter of the order-b curve is the order-(b-1) curve mirrored
    # about the diagonal; the last quarter is mirrored about the anti-diagonal
    b = 4
    s = 1 << (b - 1)
    lower = hilbert_inverse(b - 1)
    full = hilbert_inverse(b)
    q = len(lower)
    assert full[:q] == [(y, x) for (x, y) in lower]
    assert full[q:2 * q] == [(x, y + s) for (x, y) in lower]
    assert full[2 * q:3 * q] == [(x + s, y + s) for (x, y) in lower]
    assert full[3 * q:] == [(2 * s - 1 - y, s - 1 - x) for (x, y) in lower]


def test_hilbert_self_similar_at_30_bits():
    rng = np.random.default_rng(0)
    for x, y in rng.integers(0, 64, size=(300, 2)):
        assert O.hilbert2(int(x) << 24, int(y) << 24, 30) >> 48 == O.hilbert2(int(x), int(y), 6)
    # largest values stay inside 60 bits and the curve ends at (2^30-1, 0)
    assert O.hilbert2((1 << 30) - 1, 0, 30) == (1 << 60) - 1
    assert O.hilbert2(0, 0, 30) == 0


def test_hilbert_lower_left_quadrant_is_the_mirrored_curve():
    # the first quadrant of a curve of b + 1 levels is the b-level curve mirrored
    # about the diagonal (x and y exchanged), so two extra levels change nothing
    rng = np.random.default_rng(4)
    for bits in (1, 2, 5, 13, 29):
        for x, y in rng.integers(0, 1 << bits, size=(200, 2)):
            x, y = int(x), int(y)
            assert O.hilbert2(x, y, bits + 1) == O.hilbert2(y, x, bits)
            if bits + 2 <= 31:
                assert O.hilbert2(x, y, bits + 2) == O.hilbert2(x, y, bits)


def hilbert3_inverse(bits):
    side = 1 << bits
    cells = [None] * (side ** 3)
    for x in range(side):
        for y in range(side):
            for z in range(side):
                d = O.hilbert3(x, y, z, bits)
                assert 0 <= d < len(cells)
                assert cells[d] is None, "not a bijection"
                cells[d] = (x, y, z)
    return cells


def test_hilbert3_order_one_is_gray_code():
    # the first-order 3D curve visits the cube's corners in reflected binary
    # Gray-code order, x the most significant bit: g(k) = k ^ (k >> 1)
    want = [((k ^ (k >> 1)) >> 2 & 1, (k ^ (k >> 1)) >> 1 & 1, (k ^ (k >> 1)) & 1) for k in range(8)]
    assert hilbert3_inverse(1) == want


@pytest.mark.parametrize("bits", [2, 3, 4])
def test_hilbert3_bijection_adjacency_endpoints_nesting(bits):
    cells = hilbert3_inverse(bits)
    side = 1 << bits
    assert cells[0] == (0, 0, 0)
    assert cells[-1] == (side - 1, 0, 0)
    for a, b in zip(cells, cells[1:]):
        assert sum(abs(a[i] - b[i]) for i in range(3)) == 1
    # every aligned run of 8^j indices fills an aligned 2^j cube
    for j in range(1, bits):
        blk = 1 << (3 * j)
        for t in range(0, len(cells), blk):
            for axis in range(3):
                assert len({c[axis] >> j for c in cells[t:t + blk]}) == 1


def test_hilbert3_self_similar_at_21_bits():
    rng = np.random.default_rng(2)
    for x, y, z in rng.integers(0, 16, size=(300, 3)):
        top = O.hilbert3(int(x) << 17, int(y) << 17, int(z) << 17, 21)
        assert top >> 51 == O.hilbert3(int(x), int(y), int(z), 4)
    assert O.hilbert3(0, 0, 0, 21) == 0
    assert O.hilbert3((1 << 21) - 1, 0, 0, 21) == (1 << 63) - 1
    # neighbours along the curve stay neighbours at full resolution: walk the
    # keys of a small aligned cube deep inside the domain
    base = np.array([123456, 987654, 1 << 20]) & ~np.int64(7)
    cells = {}
    for dx in range(8):
        for dy in range(8):
            for dz in range(8):
                cells[O.hilbert3(int(base[0] + dx), int(base[1] + dy), int(base[2] + dz), 21)] = (dx, dy, dz)
    ks = sorted(cells)
    assert ks[-1] - ks[0] == 511  # an aligned 8^3 cube is one contiguous run
    for a, b in zip(ks, ks[1:]):
        assert sum(abs(cells[a][i] - cells[b][i]) for i in range(3)) == 1


def test_keys_reject_out_of_range():
    with pytest.raises(ValueError):
        O.keys(np.array([[1 << 30, 0]]), 2, O.SPAC_Z, 30)
    with pytest.raises(ValueError):
        O.keys(np.array([[-1, 0]]), 2, O.SPAC_Z, 30)
    with pytest.raises(ValueError):
        O.keys(np.array([[0, 0, 1 << 21]]), 3, O.PORTH, 21)


def test_keys_batch_matches_scalar():
    rng = np.random.default_rng(1)
    p = rng.integers(0, 1 << 30, size=(50, 2))
    kz = O.keys(p, 2, O.SPAC_Z, 30)
    kh = O.keys(p, 2, O.SPAC_H, 30)
    for i, (x, y) in enumerate(p):
        assert kz[i] == O.morton([x, y], 2, 30)
        assert kh[i] == O.hilbert2(x, y, 30)
    p3 = rng.integers(0, 1 << 21, size=(50, 3))
    k3 = O.keys(p3, 3, O.SPAC_H, 21)
    for i, (x, y, z) in enumerate(p3):
        assert k3[i] == O.hilbert3(x, y, z, 21)
