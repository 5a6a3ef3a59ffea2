"""Autotuner of the batched many-index form.

Chooses the leaf size (16, 32, 64), the thread-block size of the persistent
build (256, 512, 1024) and the digit width of its block sort (8 or 11 bits;
11-bit digits with 256 or 512 threads only) by timing build + k-NN on a sample
of the batch with CUDA events, and caches the choice in a JSON file keyed by
(kind, dim, size bucket, distribution).  Results do not depend on the choice:
k-NN answers are defined by the point set alone.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

from . import psi

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")
LEAF_SIZES = (16, 32, 64)
THREADS = (256, 512, 1024)
RADIX_BITS = (8, 11)


def cache_key(kind: str, dim: int, sizes: np.ndarray, dist: str) -> str:
    mean = float(np.mean(sizes)) if len(sizes) else 0.0
    return f"{kind}/{dim}d/size~2^{int(round(math.log2(max(mean, 1.0))))}/{dist}"


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d: dict):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def time_config(off, dpts, dids, dq, dqoff, nq, k, *, dim, kind, leaf_size, threads, radix_bits=8,
                reps=3) -> float:
    """Milliseconds of one batched build + k-NN pass (mean of reps after one warm-up)."""
    b = psi.Batch(off, dim=dim, kind=kind, leaf_size=leaf_size, threads=threads, radix_bits=radix_bits)
    b.reserve(nq)
    out_i = torch.empty((nq, k), dtype=torch.int32, device=dpts.device)
    out_d = torch.empty((nq, k), dtype=torch.int64, device=dpts.device)
    b.build(dpts, dids)
    b.knn(dq, dqoff, k, out_i, out_d)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        b.build(dpts, dids)
        b.knn(dq, dqoff, k, out_i, out_d)
    e1.record(s)
    torch.cuda.synchronize()
    b.close()
    return e0.elapsed_time(e1) / reps


def autotune(off, dpts, dids, dq, dqoff, nq, k, *, dim: int, kind: str, dist: str, sizes, refresh=False):
    """Best (leaf_size, threads, radix_bits) for this batch shape, from the cache or by timing."""
    key = cache_key(kind, dim, np.asarray(sizes), dist)
    cache = _load()
    if key in cache and not refresh and "radix_bits" in cache[key]:
        return cache[key]["leaf_size"], cache[key]["threads"], cache[key]["radix_bits"], cache[key]
    trials = {}
    for phi in LEAF_SIZES:
        for th in THREADS:
            for rb in RADIX_BITS:
                if rb == 11 and th == 1024:
                    continue  # 11-bit digits do not fit a 1024-thread block's shared memory
                trials[f"{phi}/{th}/{rb}"] = time_config(off, dpts, dids, dq, dqoff, nq, k, dim=dim, kind=kind,
                                                         leaf_size=phi, threads=th, radix_bits=rb)
    best = min(trials, key=trials.get)
    phi, th, rb = (int(x) for x in best.split("/"))
    cache[key] = {"leaf_size": phi, "threads": th, "radix_bits": rb, "ms": trials[best], "trials_ms": trials}
    _save(cache)
    return phi, th, rb, cache[key]
