"""The algorithmic bytes behind the bench's sort roofline: one digit pass moves
(key 8 B, value 4 B) in and out; an encoding sort of at least 2^22 locally
ordered pairs packs (position, unsorted key bits) into one 8-B word for its
middle passes.  Each figure is the per-pass sum written out by hand."""
import bench


def test_pairs_sort_of_hilbert_keys():
    # 8 passes of 60-bit keys: pass 0 reads the written key (8) and writes a pair (12),
    # seven more passes move pairs (24); the histogram pass reads the point and writes the key
    hist, passes = bench.sort_bytes(1000, 60, True)
    assert hist == 1000 * (8 + 8)
    assert passes == 1000 * (20 + 7 * 24)


def test_pairs_sort_of_morton_keys_in_3d():
    # Morton keys are not written: histogram and first pass read the 12-B point
    hist, passes = bench.sort_bytes(1000, 63, False, dim=3)
    assert hist == 1000 * 12
    assert passes == 1000 * (12 + 12 + 7 * 24)


def test_packed_sort_of_a_walk_ordered_1e8_build():
    # 27-bit positions: 27 + 60 - 8 * 3 <= 64, so pass 2 packs; passes 3..6 move words; pass 7 unpacks
    n = 100_000_000
    hist, passes = bench.sort_bytes(n, 60, True, local=True)
    assert hist == n * 16
    assert passes == n * (20 + 24 + (12 + 8) + 4 * 16 + (8 + 8 + 12))


def test_packing_needs_size_and_local_order():
    big = 1 << 22
    assert bench.sort_bytes(big, 60, True, local=False) == bench.sort_bytes(big, 60, True)
    assert bench.sort_bytes(big - 1, 60, True, local=True) == ((big - 1) * 16, (big - 1) * (20 + 7 * 24))
    _, packed = bench.sort_bytes(big, 60, True, local=True)
    assert packed < big * (20 + 7 * 24)


def test_query_order_sort_is_six_passes_of_pairs():
    # 1e7 queries in random order, top 48 key bits
    hist, passes = bench.sort_bytes(10_000_000, 48, True)
    assert passes == 10_000_000 * (20 + 5 * 24)


def test_prefix_mode_build_sorts_six_digits():
    # the top 48 of 60 key bits: pass 0 reads the written key and writes a pair (20); with
    # 27-bit positions 27 + 48 - 8 * 2 <= 64, so pass 1 packs (pairs in 12, words out 8);
    # passes 2..4 move words (16); pass 5 reads a word, gathers the key and writes a pair (28)
    n = 100_000_000
    hist, passes = bench.sort_bytes(n, 60, True, local=True, prefix=True)
    assert hist == n * 16
    assert passes == n * (20 + 20 + 3 * 16 + 28)


def test_prefix_mode_is_counted_only_when_the_build_took_it():
    w = {"n": 100_000_000, "m_ins": 1_000_000, "m_del": 1_000_000, "n_knn": 10_000_000}
    full = bench.kernel_bytes("k_onesweep", w, 28)
    pref = bench.kernel_bytes("k_onesweep", w, 26, prefix_build=True)
    assert full - pref == 100_000_000 * ((20 + 24 + 20 + 4 * 16 + 28) - (20 + 20 + 3 * 16 + 28))


def test_traffic_records_parse_and_name_their_summaries():
    import os
    path = os.path.join(bench.ROOT, "profiles", "traffic.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kernel, digest, workload, dram, lts, src = line.rstrip("\n").split("\t")[:6]
        assert kernel in bench.KERNEL_SOURCES and len(digest) == 16 and workload
        assert float(dram) > 0 and (lts == "-" or float(lts) > 0)
        assert os.path.exists(os.path.join(bench.ROOT, src))


def test_source_digest_follows_the_bytes(tmp_path, monkeypatch):
    a = tmp_path / "a.cu"
    a.write_text("x")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d1 = bench.source_digest(["a.cu"])
    a.write_text("y")
    assert bench.source_digest(["a.cu"]) != d1


def test_update_bytes_add_up():
    # a 1e6-point batch into 3.125e6 leaves touching 5e5 of them, leaves of 32, fan-out 32
    m, L, t = 1_000_000, 3_125_000, 500_000
    hist, passes = bench.sort_bytes(m, 60, True)
    want = hist + passes + 8 * (L + m) + t * 64 * 24 * 2 + m * 48 + L * 32 * 32 / 31
    assert abs(bench.update_bytes(m, L, t) - want) < 1e-3
