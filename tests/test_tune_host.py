"""The batched form's autotuner (host logic, no GPU): it times every allowed
(leaf size, block size, digit width), keeps the fastest, and answers later calls
for the same batch shape from its cache."""
import numpy as np

from paper_2601_05347_gb300 import tune


def fake_timer(times, calls):
    def time_config(off, dpts, dids, dq, dqoff, nq, k, *, dim, kind, leaf_size, threads, radix_bits=8, reps=3):
        calls.append((leaf_size, threads, radix_bits))
        return times.get((leaf_size, threads, radix_bits), 10.0)
    return time_config


def run(sizes, refresh=False, dist="varden"):
    return tune.autotune(None, None, None, None, None, 0, 10, dim=2, kind="spac_h", dist=dist, sizes=sizes,
                         refresh=refresh)


def test_searches_every_allowed_configuration_and_keeps_the_fastest(tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "cache.json"))
    calls = []
    monkeypatch.setattr(tune, "time_config", fake_timer({(64, 512, 11): 3.0, (16, 1024, 8): 4.0}, calls))
    phi, th, rb, rec = run(np.full(8, 5000))
    want = {(p, t, r) for p in tune.LEAF_SIZES for t in tune.THREADS for r in tune.RADIX_BITS
            if not (r == 11 and t == 1024)}
    assert set(calls) == want and len(calls) == len(want) == 15
    assert (phi, th, rb) == (64, 512, 11) and rec["ms"] == 3.0 and len(rec["trials_ms"]) == 15


def test_cache_answers_the_same_shape_and_refresh_retimes(tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "cache.json"))
    calls = []
    monkeypatch.setattr(tune, "time_config", fake_timer({(32, 256, 8): 1.0}, calls))
    assert run(np.full(4, 3000))[:3] == (32, 256, 8)
    n = len(calls)
    # same size bucket (mean about 2^12) and distribution: from the cache
    assert run(np.full(6, 3500))[:3] == (32, 256, 8) and len(calls) == n
    # another distribution or size bucket: timed again
    run(np.full(4, 3000), dist="uniform")
    assert len(calls) == 2 * n
    run(np.full(4, 300000))
    assert len(calls) == 3 * n
    # refresh re-times, and a changed timing changes the choice
    monkeypatch.setattr(tune, "time_config", fake_timer({(16, 512, 11): 0.5}, calls))
    assert run(np.full(4, 3000), refresh=True)[:3] == (16, 512, 11)
    assert len(calls) == 4 * n


def test_cache_entries_without_a_digit_width_are_timed_again(tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "cache.json"))
    sizes = np.full(4, 3000)
    key = tune.cache_key("spac_h", 2, sizes, "varden")
    tune._save({key: {"leaf_size": 16, "threads": 256, "ms": 1.0}})
    calls = []
    monkeypatch.setattr(tune, "time_config", fake_timer({(64, 1024, 8): 2.0}, calls))
    assert run(sizes)[:3] == (64, 1024, 8) and len(calls) == 15
