"""Seeded synthetic workloads shaped like the paper's (Sec 5.1: Uniform and Varden).

This module holds only random draws and workload shapes -- none of the index
arithmetic -- so the tests, the oracle and the CUDA path can share it.  Every
draw is SplitMix64 in counter form (Steele, Lea and Flood, OOPSLA 2014): value i
of a stream with seed s is ``mix(s + (i + 1) * 0x9E3779B97F4A7C15)`` with the
published finaliser, so any slice of any stream can be regenerated
independently and identically on any machine.

Workload recipe:
  * Uniform: each coordinate is the top ``bits`` bits of one 64-bit draw.
  * Varden (random walks, the generator of Gan and Tao 2017 as the paper uses
    it): ``clusters`` walkers each produce a contiguous share of the points;
    a walker starts at a uniform position in the region, then each point either
    restarts at a new uniform position (probability ``p_restart``) or moves by a
    step drawn uniformly from [-step, step] per coordinate.  The walk is folded
    (reflected) into the region.
  * Sweepline: the Uniform points ordered by their first coordinate (ties in
    generation order), so that consecutive batches of an incremental workload
    are spatially local strips (Sec 5.1).
  * Out-of-distribution batches for a clustered base live in the other half of
    the x range.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 outputs for the given counters (uint64 array) of stream ``seed``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + (c + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, stream: int) -> int:
    """Seed of an independent sub-stream (one SplitMix64 draw of the parent)."""
    return int(splitmix64(seed, np.array([stream], np.uint64))[0])


def config_seed(cfg_index: int, stream: int = 0, rank: int = 0) -> int:
    """Seed layout of the benchmark configurations."""
    return 0x5EED0000 + cfg_index * 256 + stream + (rank << 20)


def _uniform_below(u64: np.ndarray, width: int) -> np.ndarray:
    """Map draws to [0, width) by multiply-shift of their top 32 bits (width <= 2^32)."""
    return ((u64 >> np.uint64(32)) * np.uint64(width)) >> np.uint64(32)


def uniform(n: int, dim: int, bits: int, seed: int) -> np.ndarray:
    """n points with iid uniform int32 coordinates in [0, 2^bits)."""
    d = splitmix64(stream_seed(seed, 0), np.arange(n * dim, dtype=np.uint64))
    return (d >> np.uint64(64 - bits)).astype(np.int32).reshape(n, dim)


def sweepline(n: int, dim: int, bits: int, seed: int) -> np.ndarray:
    """The points of ``uniform(n, dim, bits, seed)`` sorted by first coordinate (stable)."""
    p = uniform(n, dim, bits, seed)
    return p[np.argsort(p[:, 0], kind="stable")]


def varden(n: int, dim: int, bits: int, seed: int, clusters: int = 100, step: int | None = None,
           p_restart: float = 1e-4, x_range: tuple[int, int] | None = None) -> np.ndarray:
    """n clustered points from ``clusters`` folded random walks (see module docstring)."""
    if step is None:
        step = 1 << 10 if dim == 2 else 1 << 4
    full = 1 << bits
    lo = [0] * dim
    width = [full] * dim
    if x_range is not None:
        lo[0], width[0] = x_range[0], x_range[1] - x_range[0]
    out = np.empty((n, dim), np.int32)
    if n == 0:
        return out
    idx = np.arange(n, dtype=np.uint64)
    walker = (np.arange(n, dtype=np.int64) * clusters) // n
    start = np.ones(n, bool)
    start[1:] = walker[1:] != walker[:-1]
    thresh = np.uint64(int(p_restart * 2.0 ** 64))
    start |= splitmix64(stream_seed(seed, 1), idx) < thresh
    seg = np.cumsum(start) - 1
    seg_first = np.flatnonzero(start)
    for d in range(dim):
        startpos = (lo[d] + _uniform_below(splitmix64(stream_seed(seed, 2 + d), idx), width[d]).astype(np.int64))
        s = _uniform_below(splitmix64(stream_seed(seed, 10 + d), idx), 2 * step + 1).astype(np.int64) - step
        s[start] = 0
        cs = np.cumsum(s)
        unbounded = startpos[seg_first][seg] + (cs - cs[seg_first][seg])
        m = width[d] - 1
        if m == 0:
            out[:, d] = lo[d]
            continue
        t = np.mod(unbounded - lo[d], 2 * m)
        t = np.where(t > m, 2 * m - t, t)
        out[:, d] = (lo[d] + t).astype(np.int32)
    return out


def sample_without_replacement(n: int, m: int, seed: int) -> np.ndarray:
    """m distinct indices from [0, n), in draw order."""
    if m > n:
        raise ValueError("m > n")
    if m == 0:
        return np.empty(0, np.int64)
    if 4 * m >= n:
        perm = np.argsort(splitmix64(seed, np.arange(n, dtype=np.uint64)), kind="stable")
        return perm[:m].astype(np.int64)
    got = np.empty(0, np.int64)
    base = 0
    while len(got) < m:
        want = 2 * (m - len(got)) + 16
        c = (splitmix64(seed, np.arange(base, base + want, dtype=np.uint64)) % np.uint64(n)).astype(np.int64)
        base += want
        allc = np.concatenate([got, c])
        _, first = np.unique(allc, return_index=True)
        got = allc[np.sort(first)]
    return got[:m]


def sample_with_replacement(n: int, m: int, seed: int) -> np.ndarray:
    return (splitmix64(seed, np.arange(m, dtype=np.uint64)) % np.uint64(max(n, 1))).astype(np.int64)


def square_boxes(q: int, dim: int, bits: int, side: int, seed: int) -> np.ndarray:
    """q axis-aligned closed boxes [lo, lo + side - 1] with lo uniform in [0, 2^bits - side)."""
    span = (1 << bits) - side
    d = splitmix64(stream_seed(seed, 0), np.arange(q * dim, dtype=np.uint64))
    lo = _uniform_below(d, span).astype(np.int64).reshape(q, dim)
    return np.concatenate([lo, lo + side - 1], axis=1).astype(np.int32)


def centred_boxes(centres: np.ndarray, half: int, bits: int) -> np.ndarray:
    """Boxes [c - half, c + half] clipped to the domain."""
    c = centres.astype(np.int64)
    lo = np.clip(c - half, 0, (1 << bits) - 1)
    hi = np.clip(c + half, 0, (1 << bits) - 1)
    return np.concatenate([lo, hi], axis=1).astype(np.int32)


def half_side_for_count(points: np.ndarray, target: float, seed: int, sample: int = 1_000_000,
                        probes: int = 256) -> int:
    """Half side h such that boxes of side 2h+1 centred on data points hold about
    ``target`` points (median over ``probes`` centres), estimated on a subsample."""
    n, dim = points.shape
    bits = int(np.ceil(np.log2(max(int(points.max()) + 1, 2))))
    take = min(n, sample)
    sub = points[sample_without_replacement(n, take, stream_seed(seed, 0))].astype(np.int64)
    order = np.argsort(sub[:, 0], kind="stable")
    sub = sub[order]
    xs = sub[:, 0]
    cen = points[sample_with_replacement(n, probes, stream_seed(seed, 1))].astype(np.int64)
    scale = n / take

    def median_count(h):
        counts = np.empty(probes)
        for i, c in enumerate(cen):
            a, b = np.searchsorted(xs, c[0] - h, "left"), np.searchsorted(xs, c[0] + h, "right")
            s = sub[a:b]
            counts[i] = np.all(np.abs(s[:, 1:] - c[1:]) <= h, axis=1).sum() * scale
        return np.median(counts)

    lo_h, hi_h = 0, 1 << bits
    for _ in range(40):
        if hi_h - lo_h <= 1:
            break
        mid = (lo_h + hi_h) // 2
        if median_count(mid) < target:
            lo_h = mid
        else:
            hi_h = mid
    return int(hi_h)
